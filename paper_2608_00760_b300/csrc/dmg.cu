// Host runtime and C ABI of the B300 multigrid solver (declared in include/dmg.h).
//
// The runtime owns the grid hierarchy (Sec. 2.2 of arXiv 2608.00760: levels
// h_k = 2 h_{k-1}, operator rediscretised per level) and schedules the kernels
// of kernels.cuh on the caller's stream: the V-cycle (Eq. 5), its transpose
// (Sec. 2.4, Eq. 18), the convergence loop, mixed-precision refinement and the
// derivative kernels. It computes nothing itself.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/dmg.h"
#include "kernels.cuh"

using dmgk::Geom;

namespace {

thread_local char g_setup_err[512];

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarse = 512;
constexpr int kNormBlocks = 148 * 4;

struct Level {
    Geom g;
    double h;
    size_t n;   // padded element count
    // FP64
    double *u = nullptr, *f = nullptr, *r = nullptr;
    double *cx = nullptr, *cy = nullptr, *cz = nullptr, *diag = nullptr, *invd = nullptr;
    double *D = nullptr, *mu = nullptr;
    // FP32 mirror (mixed precision): vertex coefficients
    float *u32 = nullptr, *f32 = nullptr, *r32 = nullptr, *Dh32 = nullptr, *mu32 = nullptr;
};

}  // namespace

struct dmg_ctx {
    dmg_params p;
    int nlev = 0;
    Level L[kMaxLevels];
    int nc = 0;                       // coarsest interior unknowns
    double *Ainv = nullptr;           // coarsest inverse (FP64)
    float *Ainv32 = nullptr;
    double *U0 = nullptr;             // level-0 staging: user's u
    double *T1 = nullptr, *T2 = nullptr, *T3 = nullptr;  // level-0 staging: tangents / outputs
    double *partial = nullptr;        // reduction partials
    double *red = nullptr;            // reduction results (device, 4 doubles)
    double *hred = nullptr;           // pinned host copy of red
    std::vector<void *> dev_allocs;
    unsigned long long launches = 0;
    char err[512] = {0};
    // profiling
    int prof_kernel = -1, prof_level = 0, prof_fp32 = 0, prof_max = 0, prof_n = 0;
    std::vector<cudaEvent_t> prof_ev;
};

namespace {

dmg_status fail(dmg_ctx *c, dmg_status s, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CUDA_TRY(ctx, call)                                                                 \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((ctx), DMG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

#define TRY(expr)                          \
    do {                                   \
        dmg_status s_ = (expr);            \
        if (s_ != DMG_OK) return s_;       \
    } while (0)

inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// interior launch: block (32, 8), grid over interior x/y, one z-plane per blockIdx.z
inline dim3 blk() { return dim3(32, 8, 1); }
inline dim3 grid_int(const Geom &g, int xdiv = 1) {
    int nxi = (g.nx - 2 + xdiv - 1) / xdiv;
    return dim3((nxi + 31) / 32, (g.ny - 2 + 7) / 8, g.nz - 2);
}
inline dim3 grid_all(const Geom &g) { return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz); }

dmg_status check_launch(dmg_ctx *c, const char *what) {
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, DMG_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return DMG_OK;
}

template <class T>
dmg_status dalloc(dmg_ctx *c, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DMG_ENOMEM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T),
                    cudaGetErrorString(e));
    }
    c->dev_allocs.push_back(q);
    *p = static_cast<T *>(q);
    return DMG_OK;
}

// --- profiling hooks -------------------------------------------------------
struct ProfScope {
    dmg_ctx *c;
    cudaStream_t s;
    bool on;
    ProfScope(dmg_ctx *c_, int kernel, int level, int fp32, cudaStream_t s_) : c(c_), s(s_) {
        on = c->prof_kernel == kernel && c->prof_level == level && c->prof_fp32 == fp32 &&
             c->prof_n < c->prof_max;
        if (on) cudaEventRecord(c->prof_ev[2 * c->prof_n], s);
    }
    ~ProfScope() {
        if (on) {
            cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], s);
            c->prof_n++;
        }
    }
};

// --- staging between the caller's contiguous arrays and the padded layout ---
dmg_status stage_in(dmg_ctx *c, const double *src, double *dst, cudaStream_t s) {
    const Geom &g = c->L[0].g;
    CUDA_TRY(c, cudaMemcpy2DAsync(dst, (size_t)g.sy * sizeof(double), src, (size_t)g.nx * sizeof(double),
                                  (size_t)g.nx * sizeof(double), (size_t)g.ny * g.nz, cudaMemcpyDefault, s));
    return DMG_OK;
}

dmg_status stage_out(dmg_ctx *c, const double *src, double *dst, cudaStream_t s) {
    const Geom &g = c->L[0].g;
    CUDA_TRY(c, cudaMemcpy2DAsync(dst, (size_t)g.nx * sizeof(double), src, (size_t)g.sy * sizeof(double),
                                  (size_t)g.nx * sizeof(double), (size_t)g.ny * g.nz, cudaMemcpyDefault, s));
    return DMG_OK;
}

// zero the boundary of a padded level-0 FP64 array that was staged from the caller
dmg_status zero_boundary(dmg_ctx *c, double *x, cudaStream_t s) {
    const Geom &g = c->L[0].g;
    size_t row = (size_t)g.sy * sizeof(double);
    // planes k = 0 and k = nz-1
    CUDA_TRY(c, cudaMemsetAsync(x, 0, (size_t)g.sz * sizeof(double), s));
    CUDA_TRY(c, cudaMemsetAsync(x + (size_t)(g.nz - 1) * g.sz, 0, (size_t)g.sz * sizeof(double), s));
    // rows j = 0 and j = ny-1 of every plane; columns i = 0 and i = nx-1 of every row
    CUDA_TRY(c, cudaMemset2DAsync(x, (size_t)g.sz * sizeof(double), 0, row, g.nz, s));
    CUDA_TRY(c, cudaMemset2DAsync(x + (size_t)(g.ny - 1) * g.sy, (size_t)g.sz * sizeof(double), 0, row, g.nz, s));
    CUDA_TRY(c, cudaMemset2DAsync(x, row, 0, sizeof(double), (size_t)g.ny * g.nz, s));
    CUDA_TRY(c, cudaMemset2DAsync(x + (g.nx - 1), row, 0, sizeof(double), (size_t)g.ny * g.nz, s));
    return DMG_OK;
}

// --- coefficient policies per level -----------------------------------------
inline dmgk::FaceCoef<double> coef64(const Level &l) {
    return dmgk::FaceCoef<double>{l.cx, l.cy, l.cz, l.diag, l.invd};
}

// --- kernels on one level ------------------------------------------------------
template <class T> T *U(Level &l);
template <> double *U<double>(Level &l) { return l.u; }
template <> float *U<float>(Level &l) { return l.u32; }
template <class T> T *F(Level &l);
template <> double *F<double>(Level &l) { return l.f; }
template <> float *F<float>(Level &l) { return l.f32; }
template <class T> T *R(Level &l);
template <> double *R<double>(Level &l) { return l.r; }
template <> float *R<float>(Level &l) { return l.r32; }
template <class T> T *AINV(dmg_ctx *c);
template <> double *AINV<double>(dmg_ctx *c) { return c->Ainv; }
template <> float *AINV<float>(dmg_ctx *c) { return c->Ainv32; }

template <class Fn>
dmg_status with_coef32(dmg_ctx *c, Level &l, Fn fn) {
    if (c->p.face_mean == DMG_FACE_HARMONIC) return fn(dmgk::VertCoef<float, true>{l.Dh32, l.mu32});
    return fn(dmgk::VertCoef<float, false>{l.Dh32, l.mu32});
}

template <class T, class Fn>
dmg_status dispatch(dmg_ctx *c, Level &l, Fn fn) {
    if constexpr (sizeof(T) == 8) return fn(coef64(l));
    else return with_coef32(c, l, fn);
}

// nsweeps RB-GS sweeps; each sweep is the half-sweep of colour `first` then the other
template <class T>
dmg_status smooth(dmg_ctx *c, int lev, int first, int nsweeps, cudaStream_t s) {
    Level &l = c->L[lev];
    for (int it = 0; it < nsweeps; it++) {
        ProfScope ps(c, DMG_KERNEL_SMOOTH, lev, sizeof(T) == 4, s);
        for (int h = 0; h < 2; h++) {
            int color = h == 0 ? first : 1 - first;
            TRY(dispatch<T>(c, l, [&](auto cf) {
                dmgk::k_smooth_half<T><<<grid_int(l.g, 2), blk(), 0, s>>>(l.g, U<T>(l), F<T>(l), cf, color);
                return check_launch(c, "smooth");
            }));
        }
    }
    return DMG_OK;
}

// f_{l+1} = R (f_l - A_l u_l), u_{l+1} = 0
template <class T>
dmg_status restrict_defect(dmg_ctx *c, int lev, cudaStream_t s) {
    Level &l = c->L[lev], &cl = c->L[lev + 1];
    ProfScope ps(c, DMG_KERNEL_RESTRICT, lev, sizeof(T) == 4, s);
    TRY(dispatch<T>(c, l, [&](auto cf) {
        dmgk::k_residual<T><<<grid_int(l.g), blk(), 0, s>>>(l.g, U<T>(l), F<T>(l), cf, R<T>(l));
        return check_launch(c, "residual");
    }));
    dmgk::k_restrict<T><<<grid_int(cl.g), blk(), 0, s>>>(l.g, R<T>(l), cl.g, F<T>(cl));
    TRY(check_launch(c, "restrict"));
    CUDA_TRY(c, cudaMemsetAsync(U<T>(cl), 0, cl.n * sizeof(T), s));
    return DMG_OK;
}

template <class T>
dmg_status prolong(dmg_ctx *c, int lev, cudaStream_t s) {
    Level &l = c->L[lev], &cl = c->L[lev + 1];
    ProfScope ps(c, DMG_KERNEL_PROLONG, lev, sizeof(T) == 4, s);
    dmgk::k_prolong_add<T><<<grid_int(l.g), blk(), 0, s>>>(cl.g, U<T>(cl), l.g, U<T>(l));
    return check_launch(c, "prolong");
}

template <class T>
dmg_status coarse_solve(dmg_ctx *c, cudaStream_t s) {
    Level &l = c->L[c->nlev - 1];
    int threads = c->nc < 32 ? 32 : (c->nc > 512 ? 512 : ((c->nc + 31) / 32) * 32);
    dmgk::k_coarse_solve<T><<<1, threads, c->nc * sizeof(T), s>>>(l.g, AINV<T>(c), c->nc, F<T>(l), U<T>(l));
    return check_launch(c, "coarse_solve");
}

// One V-cycle at level lev on (u_lev, f_lev), in place (Sec. 2.2, Fig. 1 left).
// transposed: the V-cycle whose preconditioner is the transpose of the forward
// one (Sec. 2.4): nu2 pre-sweeps and nu1 post-sweeps, colour orders reversed.
template <class T>
dmg_status vcycle(dmg_ctx *c, int lev, bool transposed, cudaStream_t s) {
    if (lev == c->nlev - 1) return coarse_solve<T>(c, s);
    int post_first = c->p.symmetric ? 1 : 0;
    int npre = transposed ? c->p.nu2 : c->p.nu1, npost = transposed ? c->p.nu1 : c->p.nu2;
    int pre_first = transposed ? 1 - post_first : 0;
    int postf = transposed ? 1 : post_first;
    TRY(smooth<T>(c, lev, pre_first, npre, s));
    TRY(restrict_defect<T>(c, lev, s));
    TRY(vcycle<T>(c, lev + 1, transposed, s));
    TRY(prolong<T>(c, lev, s));
    TRY(smooth<T>(c, lev, postf, npost, s));
    return DMG_OK;
}

// --- reductions ------------------------------------------------------------------
dmg_status finish_reduce(dmg_ctx *c, int nslots, cudaStream_t s, double *out) {
    CUDA_TRY(c, cudaMemcpyAsync(c->hred, c->red, nslots * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    for (int i = 0; i < nslots; i++) out[i] = c->hred[i];
    return DMG_OK;
}

// ||x||_2^2 over interior of a level-0 FP64 array -> red[slot]
dmg_status norm2_async(dmg_ctx *c, const double *x, int slot, cudaStream_t s) {
    dmgk::k_norm2<<<kNormBlocks, 256, 0, s>>>(c->L[0].g, x, c->partial);
    TRY(check_launch(c, "norm2"));
    dmgk::k_reduce_final<<<1, 256, 0, s>>>(c->partial, kNormBlocks, c->red, slot);
    return check_launch(c, "reduce");
}

// ||f - A u||^2 (FP64, level 0) -> red[slot]; optional r32 = (r * r32_scale)
dmg_status resid_norm_async(dmg_ctx *c, const double *u, const double *f, float *r32, double r32_scale,
                            int slot, cudaStream_t s) {
    Level &l = c->L[0];
    {
        ProfScope ps(c, DMG_KERNEL_RESIDUAL, 0, 0, s);
        dmgk::k_resid_norm<double><<<kNormBlocks, 256, 0, s>>>(l.g, u, f, coef64(l), (double *)nullptr, r32,
                                                               r32_scale, c->partial);
        TRY(check_launch(c, "resid_norm"));
    }
    dmgk::k_reduce_final<<<1, 256, 0, s>>>(c->partial, kNormBlocks, c->red, slot);
    return check_launch(c, "reduce");
}

void info_reset(dmg_info *info) {
    if (!info) return;
    memset(info, 0, sizeof(*info));
}

// Plain FP64 iteration on level 0: u_0 = 0, then V-cycles on A u_0 = f_0.
// fixed > 0: exactly `fixed` cycles; else until rtol or max_cycles.
dmg_status iterate64(dmg_ctx *c, bool transposed, int fixed, dmg_info *info, cudaStream_t s) {
    Level &l = c->L[0];
    CUDA_TRY(c, cudaMemsetAsync(l.u, 0, l.n * sizeof(double), s));
    double nf2;
    TRY(norm2_async(c, l.f, 0, s));
    TRY(finish_reduce(c, 1, s, &nf2));
    if (!std::isfinite(nf2)) return fail(c, DMG_ENAN, "right-hand side is not finite");
    double nf = std::sqrt(nf2);
    if (info) { info->cycles = 0; info->outer = 0; info->rel_residual = 0.0; }
    if (nf == 0.0) return DMG_OK;
    int ncyc = fixed > 0 ? fixed : c->p.max_cycles;
    double rel = 1.0;
    int cyc = 0;
    for (cyc = 1; cyc <= ncyc; cyc++) {
        TRY(vcycle<double>(c, 0, transposed, s));
        if (fixed > 0 && cyc < ncyc) continue;
        double rn2;
        TRY(resid_norm_async(c, l.u, l.f, nullptr, 0.0, 0, s));
        TRY(finish_reduce(c, 1, s, &rn2));
        if (!std::isfinite(rn2)) return fail(c, DMG_ENAN, "residual norm is not finite after cycle %d", cyc);
        rel = std::sqrt(rn2) / nf;
        if (info && fixed == 0 && cyc - 1 < DMG_HIST_LEN) info->hist[cyc - 1] = rel;
        if (fixed == 0 && rel <= c->p.rtol) break;
    }
    if (cyc > ncyc) cyc = ncyc;
    if (info) { info->cycles = cyc; info->outer = cyc; info->rel_residual = rel; }
    if (fixed == 0 && rel > c->p.rtol)
        return fail(c, DMG_ENOCONV, "relative residual %.3e > rtol %.3e after %d cycles", rel, c->p.rtol, cyc);
    return DMG_OK;
}

// Mixed precision defect correction on level 0 (FP64 u_0, f_0): each step runs
// inner_cycles FP32 V-cycles on A e = r / scale and updates u_0 += scale * e in
// FP64; residual, norms and update stay in FP64.
dmg_status iterate_mixed(dmg_ctx *c, bool transposed, dmg_info *info, cudaStream_t s) {
    Level &l = c->L[0];
    CUDA_TRY(c, cudaMemsetAsync(l.u, 0, l.n * sizeof(double), s));
    double nf2;
    TRY(norm2_async(c, l.f, 0, s));
    TRY(finish_reduce(c, 1, s, &nf2));
    if (!std::isfinite(nf2)) return fail(c, DMG_ENAN, "right-hand side is not finite");
    double nf = std::sqrt(nf2);
    if (info) { info->cycles = 0; info->outer = 0; info->rel_residual = 0.0; }
    if (nf == 0.0) return DMG_OK;
    double scale = nf;                 // divisor carried by the FP32 right-hand side
    dmgk::k_to_f32<<<grid_int(l.g), blk(), 0, s>>>(l.g, l.f, 1.0 / scale, l.f32);
    TRY(check_launch(c, "to_f32"));
    double last = nf, rel = 1.0;
    int step = 0, inner = 0;
    for (step = 1; step <= c->p.max_cycles; step++) {
        CUDA_TRY(c, cudaMemsetAsync(l.u32, 0, l.n * sizeof(float), s));
        for (int ic = 0; ic < c->p.inner_cycles; ic++) {
            TRY(vcycle<float>(c, 0, transposed, s));
            inner++;
        }
        dmgk::k_update<<<grid_int(l.g), blk(), 0, s>>>(l.g, l.u, l.u32, scale);
        TRY(check_launch(c, "update"));
        double rn2;
        TRY(resid_norm_async(c, l.u, l.f, l.f32, 1.0 / last, 0, s));
        TRY(finish_reduce(c, 1, s, &rn2));
        if (!std::isfinite(rn2)) return fail(c, DMG_ENAN, "residual norm is not finite after step %d", step);
        scale = last;
        last = std::sqrt(rn2);
        rel = last / nf;
        if (info && step - 1 < DMG_HIST_LEN) info->hist[step - 1] = rel;
        if (rel <= c->p.rtol) break;
        if (last == 0.0) break;
    }
    if (step > c->p.max_cycles) step = c->p.max_cycles;
    if (info) { info->cycles = inner; info->outer = step; info->rel_residual = rel; }
    if (rel > c->p.rtol)
        return fail(c, DMG_ENOCONV, "relative residual %.3e > rtol %.3e after %d steps", rel, c->p.rtol, step);
    return DMG_OK;
}

dmg_status iterate(dmg_ctx *c, bool transposed, int fixed, dmg_info *info, cudaStream_t s) {
    if (fixed > 0 || c->p.precision == DMG_FP64) return iterate64(c, transposed, fixed, info, s);
    return iterate_mixed(c, transposed, info, s);
}

int count_levels(int nx, int ny, int nz) {
    if (nx < 3 || ny < 3 || nz < 3) return 0;
    int n = 1;
    while (nx > 3 && ny > 3 && nz > 3 && (nx & 1) && (ny & 1) && (nz & 1)) {
        nx = (nx - 1) / 2 + 1;
        ny = (ny - 1) / 2 + 1;
        nz = (nz - 1) / 2 + 1;
        if (++n > kMaxLevels) return 0;
    }
    return n;
}

Geom make_geom(int nx, int ny, int nz) {
    Geom g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.sy = ((nx + 31) / 32) * 32;
    g.sz = (long long)g.sy * ny;
    return g;
}

dmg_status validate(dmg_ctx *c, const dmg_params *p) {
    if (!p) return fail(c, DMG_EINVAL, "params is NULL");
    if (p->nx < 3 || p->ny < 3 || p->nz < 3)
        return fail(c, DMG_EINVAL, "grid %dx%dx%d: every axis needs >= 3 vertices", p->nx, p->ny, p->nz);
    if ((long long)p->nx * p->ny * p->nz > (1LL << 31) - 1)
        return fail(c, DMG_EINVAL, "grid %dx%dx%d too large", p->nx, p->ny, p->nz);
    if (!(p->h > 0.0) || !std::isfinite(p->h)) return fail(c, DMG_EINVAL, "h must be > 0");
    if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 < 1 || p->nu1 > 64 || p->nu2 > 64)
        return fail(c, DMG_EINVAL, "nu1, nu2 must be in [0, 64] with nu1 + nu2 >= 1");
    if (p->max_cycles < 1) return fail(c, DMG_EINVAL, "max_cycles must be >= 1");
    if (p->fixed_cycles < 0) return fail(c, DMG_EINVAL, "fixed_cycles must be >= 0");
    if (p->fixed_cycles == 0 && !(p->rtol > 0.0)) return fail(c, DMG_EINVAL, "rtol must be > 0");
    if (p->precision != DMG_FP64 && p->precision != DMG_MIXED) return fail(c, DMG_EINVAL, "bad precision");
    if (p->face_mean != DMG_FACE_ARITHMETIC && p->face_mean != DMG_FACE_HARMONIC)
        return fail(c, DMG_EINVAL, "bad face_mean");
    if (p->coarsen != DMG_COARSEN_FULL_WEIGHTING && p->coarsen != DMG_COARSEN_INJECTION)
        return fail(c, DMG_EINVAL, "bad coarsen");
    if (p->inner_cycles < 1 || p->inner_cycles > 16) return fail(c, DMG_EINVAL, "inner_cycles must be in [1, 16]");
    if (p->symmetric != 0 && p->symmetric != 1) return fail(c, DMG_EINVAL, "symmetric must be 0 or 1");
    int nl = count_levels(p->nx, p->ny, p->nz);
    if (nl == 0) return fail(c, DMG_EINVAL, "grid %dx%dx%d cannot be coarsened", p->nx, p->ny, p->nz);
    int cx = p->nx, cy = p->ny, cz = p->nz;
    for (int l = 1; l < nl; l++) { cx = (cx - 1) / 2 + 1; cy = (cy - 1) / 2 + 1; cz = (cz - 1) / 2 + 1; }
    long long nc = (long long)(cx - 2) * (cy - 2) * (cz - 2);
    if (nc > kMaxCoarse)
        return fail(c, DMG_EINVAL,
                    "grid %dx%dx%d coarsens to %dx%dx%d with %lld unknowns (> %d): use c*2^n+1 vertices with small c",
                    p->nx, p->ny, p->nz, cx, cy, cz, nc, kMaxCoarse);
    return DMG_OK;
}

dmg_status setup_impl(dmg_ctx *c, const dmg_params *p, const double *D, const double *mu, cudaStream_t s) {
    TRY(validate(c, p));
    if (!D || !mu) return fail(c, DMG_EINVAL, "D and mu must not be NULL");
    c->p = *p;
    c->nlev = count_levels(p->nx, p->ny, p->nz);
    bool mixed = p->precision == DMG_MIXED;
    for (int l = 0; l < c->nlev; l++) {
        Level &L = c->L[l];
        if (l == 0) {
            L.g = make_geom(p->nx, p->ny, p->nz);
            L.h = p->h;
        } else {
            const Level &F = c->L[l - 1];
            L.g = make_geom((F.g.nx - 1) / 2 + 1, (F.g.ny - 1) / 2 + 1, (F.g.nz - 1) / 2 + 1);
            L.h = 2.0 * F.h;
        }
        L.n = (size_t)L.g.sz * L.g.nz;
        double **f64[] = {&L.u, &L.f, &L.r, &L.cx, &L.cy, &L.cz, &L.diag, &L.invd, &L.D, &L.mu};
        for (double **q : f64) {
            TRY(dalloc(c, q, L.n));
            CUDA_TRY(c, cudaMemsetAsync(*q, 0, L.n * sizeof(double), s));
        }
        if (mixed) {
            float **f32[] = {&L.u32, &L.f32, &L.r32, &L.Dh32, &L.mu32};
            for (float **q : f32) {
                TRY(dalloc(c, q, L.n));
                CUDA_TRY(c, cudaMemsetAsync(*q, 0, L.n * sizeof(float), s));
            }
        }
    }
    Level &L0 = c->L[0];
    for (double **q : {&c->U0, &c->T1, &c->T2, &c->T3}) {
        TRY(dalloc(c, q, L0.n));
        CUDA_TRY(c, cudaMemsetAsync(*q, 0, L0.n * sizeof(double), s));
    }
    TRY(dalloc(c, &c->partial, kNormBlocks));
    TRY(dalloc(c, &c->red, 4));
    {
        cudaError_t e = cudaMallocHost(&c->hred, 4 * sizeof(double));
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, DMG_ENOMEM, "cudaMallocHost failed"); }
    }
    // level-0 coefficients from the caller, then coarsen level by level
    TRY(stage_in(c, D, L0.D, s));
    TRY(stage_in(c, mu, L0.mu, s));
    for (int l = 1; l < c->nlev; l++) {
        Level &F = c->L[l - 1], &C = c->L[l];
        dmgk::k_coarsen<<<grid_all(C.g), blk(), 0, s>>>(F.g, F.D, C.g, C.D, p->coarsen);
        TRY(check_launch(c, "coarsen"));
        dmgk::k_coarsen<<<grid_all(C.g), blk(), 0, s>>>(F.g, F.mu, C.g, C.mu, p->coarsen);
        TRY(check_launch(c, "coarsen"));
    }
    int harm = p->face_mean == DMG_FACE_HARMONIC;
    for (int l = 0; l < c->nlev; l++) {
        Level &L = c->L[l];
        double ih2 = 1.0 / (L.h * L.h);
        dmgk::k_build_faces<<<grid_all(L.g), blk(), 0, s>>>(L.g, L.D, L.mu, ih2, harm, L.cx, L.cy, L.cz,
                                                            L.diag, L.invd);
        TRY(check_launch(c, "build_faces"));
        if (mixed) {
            double scale = harm ? ih2 : 0.5 * ih2;
            dmgk::k_build_vertex32<<<grid_all(L.g), blk(), 0, s>>>(L.g, L.D, L.mu, scale, L.Dh32, L.mu32);
            TRY(check_launch(c, "build_vertex32"));
        }
    }
    // exact coarsest solve: dense SPD inverse by in-block Gauss-Jordan
    Level &LC = c->L[c->nlev - 1];
    c->nc = (LC.g.nx - 2) * (LC.g.ny - 2) * (LC.g.nz - 2);
    double *M = nullptr;
    int *status = nullptr;
    TRY(dalloc(c, &M, (size_t)c->nc * 2 * c->nc));
    TRY(dalloc(c, &c->Ainv, (size_t)c->nc * c->nc));
    TRY(dalloc(c, &c->Ainv32, (size_t)c->nc * c->nc));
    TRY(dalloc(c, &status, 1));
    CUDA_TRY(c, cudaMemsetAsync(status, 0xff, sizeof(int), s));
    dmgk::k_coarse_assemble<<<64, 256, 0, s>>>(LC.g, coef64(LC), c->nc, M);
    TRY(check_launch(c, "coarse_assemble"));
    dmgk::k_gauss_jordan<<<1, 1024, 0, s>>>(M, c->nc, c->Ainv, c->Ainv32, status);
    TRY(check_launch(c, "gauss_jordan"));
    int hstatus = -1;
    CUDA_TRY(c, cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (hstatus != 0)
        return fail(c, DMG_EINVAL, "coarsest-level matrix is not positive definite (need D > 0, mu >= 0)");
    return DMG_OK;
}

template <class F>
dmg_status guarded(dmg_ctx *c, F fn) {
    if (!c) return DMG_EINVAL;
    c->err[0] = 0;
    return fn();
}

}  // namespace

// Sets the message dmg_last_error(NULL) returns on this thread; used by the
// context-free entry point in noalloc.cu.
void dmg_detail_set_noctx_error(const char *msg) { snprintf(g_setup_err, sizeof(g_setup_err), "%s", msg); }

// ==================================================================================
// C ABI

extern "C" {

void dmg_default_params(dmg_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nu1 = 2;
    p->nu2 = 2;
    p->symmetric = 0;
    p->max_cycles = 100;
    p->rtol = 1e-10;
    p->fixed_cycles = 0;
    p->precision = DMG_FP64;
    p->face_mean = DMG_FACE_ARITHMETIC;
    p->coarsen = DMG_COARSEN_FULL_WEIGHTING;
    p->inner_cycles = 1;
}

dmg_status dmg_setup(const dmg_params *p, const double *D, const double *mu, void *stream, dmg_ctx **out) {
    if (!out) return DMG_EINVAL;
    *out = nullptr;
    dmg_ctx *c = new (std::nothrow) dmg_ctx();
    if (!c) return DMG_ENOMEM;
    dmg_status st = setup_impl(c, p, D, mu, S(stream));
    if (st != DMG_OK) {
        memcpy(g_setup_err, c->err, sizeof(g_setup_err));
        dmg_destroy(c);
        return st;
    }
    g_setup_err[0] = 0;
    *out = c;
    return DMG_OK;
}

dmg_status dmg_solve(dmg_ctx *c, const double *q, double *u, dmg_info *info, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        if (!q || !u) return fail(c, DMG_EINVAL, "q and u must not be NULL");
        info_reset(info);
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        TRY(stage_in(c, q, l.f, s));
        dmg_status st = iterate(c, false, c->p.fixed_cycles, info, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return st;
        TRY(stage_out(c, l.u, u, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        return st;
    });
}

dmg_status dmg_jvp(dmg_ctx *c, const double *u, const double *dq, const double *dD, const double *dmu,
                   double *du, dmg_info *info, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        if (!du) return fail(c, DMG_EINVAL, "du must not be NULL");
        if ((dD || dmu) && !u) return fail(c, DMG_EINVAL, "u is needed for a D or mu tangent");
        info_reset(info);
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        if (dq) {
            TRY(stage_in(c, dq, l.f, s));
        } else {
            CUDA_TRY(c, cudaMemsetAsync(l.f, 0, l.n * sizeof(double), s));
        }
        if (dD || dmu) {
            TRY(stage_in(c, u, c->U0, s));
            TRY(zero_boundary(c, c->U0, s));
            if (dD) TRY(stage_in(c, dD, c->T1, s));
            if (dmu) TRY(stage_in(c, dmu, c->T2, s));
            double ih2 = 1.0 / (l.h * l.h);
            dmgk::k_dA<<<grid_int(l.g), blk(), 0, s>>>(l.g, c->U0, dD ? c->T1 : nullptr, dmu ? c->T2 : nullptr,
                                                       l.D, ih2, c->p.face_mean == DMG_FACE_HARMONIC, l.f);
            TRY(check_launch(c, "dA"));
        }
        dmg_status st = iterate(c, false, c->p.fixed_cycles, info, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return st;
        TRY(stage_out(c, l.u, du, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        return st;
    });
}

dmg_status dmg_vjp(dmg_ctx *c, const double *u, const double *w, int cycles, double *qbar, double *Dbar,
                   double *mubar, dmg_info *info, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        if (!w) return fail(c, DMG_EINVAL, "w must not be NULL");
        if ((Dbar || mubar) && !u) return fail(c, DMG_EINVAL, "u is needed for Dbar / mubar");
        if (cycles < 0) return fail(c, DMG_EINVAL, "cycles must be >= 0");
        info_reset(info);
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        TRY(stage_in(c, w, l.f, s));
        dmg_status st = iterate(c, true, cycles, info, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return st;
        if (qbar) TRY(stage_out(c, l.u, qbar, s));
        if (Dbar || mubar) {
            TRY(stage_in(c, u, c->U0, s));
            TRY(zero_boundary(c, c->U0, s));
            double ih2 = 1.0 / (l.h * l.h);
            {
                ProfScope ps(c, DMG_KERNEL_GRAD, 0, 0, s);
                dmgk::k_grad<<<grid_all(l.g), blk(), 0, s>>>(l.g, c->U0, l.u, l.D, ih2,
                                                             c->p.face_mean == DMG_FACE_HARMONIC,
                                                             Dbar ? c->T1 : nullptr, mubar ? c->T2 : nullptr);
                TRY(check_launch(c, "grad"));
            }
            if (Dbar) TRY(stage_out(c, c->T1, Dbar, s));
            if (mubar) TRY(stage_out(c, c->T2, mubar, s));
        }
        CUDA_TRY(c, cudaStreamSynchronize(s));
        return st;
    });
}

dmg_status dmg_residual(dmg_ctx *c, const double *q, const double *u, double *out, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        if (!q || !u || !out) return fail(c, DMG_EINVAL, "q, u and out must not be NULL");
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        TRY(stage_in(c, q, c->T3, s));
        TRY(stage_in(c, u, c->U0, s));
        TRY(zero_boundary(c, c->U0, s));
        TRY(resid_norm_async(c, c->U0, c->T3, nullptr, 0.0, 0, s));
        TRY(norm2_async(c, c->T3, 1, s));
        double r[2];
        TRY(finish_reduce(c, 2, s, r));
        (void)l;
        out[0] = std::sqrt(r[0]);
        out[1] = std::sqrt(r[1]);
        return DMG_OK;
    });
}

dmg_status dmg_destroy(dmg_ctx *c) {
    if (!c) return DMG_OK;
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    for (void *q : c->dev_allocs) cudaFree(q);
    if (c->hred) cudaFreeHost(c->hred);
    delete c;
    return DMG_OK;
}

const char *dmg_strerror(dmg_status s) {
    switch (s) {
        case DMG_OK: return "ok";
        case DMG_EINVAL: return "invalid argument";
        case DMG_ENOMEM: return "out of memory";
        case DMG_ECUDA: return "CUDA error";
        case DMG_ENOCONV: return "did not converge";
        case DMG_ENAN: return "non-finite residual";
        case DMG_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char *dmg_last_error(const dmg_ctx *c) {
    if (!c) return g_setup_err;
    return c->err;
}

int dmg_levels(const dmg_ctx *c) { return c ? c->nlev : 0; }

dmg_status dmg_level_shape(const dmg_ctx *c, int level, int *nx, int *ny, int *nz) {
    if (!c || level < 0 || level >= c->nlev) return DMG_EINVAL;
    if (nx) *nx = c->L[level].g.nx;
    if (ny) *ny = c->L[level].g.ny;
    if (nz) *nz = c->L[level].g.nz;
    return DMG_OK;
}

unsigned long long dmg_launch_count(const dmg_ctx *c) { return c ? c->launches : 0; }

dmg_status dmg_profile_begin(dmg_ctx *c, int kernel, int level, int precision_fp32, int max_launches) {
    if (!c || max_launches < 1 || level < 0 || level >= c->nlev) return DMG_EINVAL;
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.assign(2 * (size_t)max_launches, nullptr);
    for (auto &e : c->prof_ev) CUDA_TRY(c, cudaEventCreate(&e));
    c->prof_kernel = kernel;
    c->prof_level = level;
    c->prof_fp32 = precision_fp32 ? 1 : 0;
    c->prof_max = max_launches;
    c->prof_n = 0;
    return DMG_OK;
}

dmg_status dmg_profile_end(dmg_ctx *c, long long *launches, double *total_ms) {
    if (!c) return DMG_EINVAL;
    double tot = 0.0;
    for (int i = 0; i < c->prof_n; i++) {
        CUDA_TRY(c, cudaEventSynchronize(c->prof_ev[2 * i + 1]));
        float ms = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
        tot += ms;
    }
    if (launches) *launches = c->prof_n;
    if (total_ms) *total_ms = tot;
    c->prof_kernel = -1;
    c->prof_n = 0;
    return DMG_OK;
}

}  // extern "C"
