// Host runtime and C ABI of the B300 multigrid solver (declared in include/dmg.h).
//
// The runtime owns the grid hierarchy (Sec. 2.2 of arXiv 2608.00760: levels
// h_k = 2 h_{k-1}, operator rediscretised per level) and schedules the kernels
// on the caller's stream: the V-cycle (Eq. 5), its transpose (Sec. 2.4,
// Eq. 18), the convergence loop, mixed-precision refinement and the derivative
// kernels (kernels.cuh; 2D grids: kernels2d.cuh; the unrolled gradient:
// unrolled.cuh). Around them: batches of independent problems, the slot-level
// serving interface, CUDA graphs per step, the tile autotuner and the
// response operator. It computes nothing itself.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dmg.h"
#include "kernels.cuh"
#include "unrolled.cuh"
#include "kernels2d.cuh"

using dmgk::Geom;

namespace {

thread_local char g_setup_err[512];

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarse = 512;
constexpr int kNormBlocks = 148 * 4;
// Levels this small run in the single-CTA tail. One SM issues 2 FP64 FMA per
// clock, so the FP64 tail starts lower than the FP32 one.
constexpr long long kTailMaxInterior[2] = {512, 4096};
constexpr size_t kTailSmemBudget = 200 * 1024;

// ceil(2^32 / d) for dmgk::mdiv (0 for d <= 1)
inline unsigned magic_div(int d) {
    return d <= 1 ? 0u : (unsigned)(((1ULL << 32) + (unsigned long long)d - 1) / (unsigned long long)d);
}

inline dmgk::TailDiv tail_div(const Geom &g) {
    return dmgk::TailDiv{magic_div(g.nx), magic_div(g.ny), magic_div(g.nx - 2), magic_div(g.ny - 2),
                         magic_div(g.nx - 1), magic_div(g.ny - 1)};
}

// unpadded split-row geometry of a level staged in shared memory
inline Geom smem_geom(const Geom &g) {
    Geom s = g;
    s.hx = g.nhalf();
    s.sy = 2 * s.hx;
    s.sz = (long long)s.sy * g.ny;
    s.sb = s.sz * g.nz;   // the staged array's extent (the tail shifts global pointers by g.sb)
    s.nb = 1;
    return s;
}

struct Level {
    Geom g;
    double h;
    size_t n;   // padded element count of all samples (nb * g.sb)
    // FP64
    double *u = nullptr, *f = nullptr, *r = nullptr;
    double *cx = nullptr, *cy = nullptr, *cz = nullptr, *diag = nullptr, *invd = nullptr;
    double *D = nullptr, *mu = nullptr;
    // FP32 mirror (mixed precision): vertex coefficients
    float *u32 = nullptr, *f32 = nullptr, *r32 = nullptr, *Dh32 = nullptr, *mu32 = nullptr;
};

// an instantiated CUDA graph, the kernels one replay launches, and the profiling
// event pairs each replay records
struct Graph {
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;
    std::vector<int> prof;
};

// Work buffers of the unrolled gradient on one level: cotangents of u and f,
// face cotangents (x, y, z faces at their lower vertex), mu and D cotangents, a
// scratch field, and the states after every half-sweep of one V-cycle (plus
// the entry state when there is no pre-smoothing).
struct ULevel {
    double *ub = nullptr, *fb = nullptr, *bx = nullptr, *by = nullptr, *bz = nullptr;
    double *mub = nullptr, *Db = nullptr, *tmp = nullptr;
    std::vector<double *> st;
};

// Host-side state of one slot of the slot-level (serving) interface.
enum SlotRun { kIdle = 0, kStarting = 1, kRunning = 2, kDone = 3 };
struct Slot {
    int phase = -1;          // DMG_PHASE_* of the current or last phase
    int run = kIdle;
    int status = DMG_OK;     // result of the last phase
    int steps = 0;           // refinement steps (mixed) or cycles (FP64) of the phase
    double nf = 0.0, rel = 0.0;
    bool start_seen = false; // its start was enqueued before the last step launch
    bool in_step = false;    // it iterated in the last step launch
    bool load_pending = false;
    bool load_failed = false;
    bool loaded = false;
    bool have_fwd = false;   // U0 holds the slot's forward solution
};

}  // namespace

struct dmg_ctx {
    dmg_params p;
    int dim = 3;                      // 3, or 2 for an (ny, nx) grid (nz == 1)
    int nb = 1;                       // samples in the batch
    // thread-block shape of the colour kernels (half-sweep, colour defect) per
    // level: [0] FP64, [1] FP32; 32 x 8 (FP64) and, FP32 (two vertices per
    // thread), 32 x 4 / 16 x 8 / 8 x 16 by the level's width, unless the
    // autotuner chose another
    dim3 tb[2][kMaxLevels];
    int nlev = 0;
    Level L[kMaxLevels];
    int nc = 0;                       // coarsest interior unknowns
    int tail_first[2] = {0, 0};       // first level of the single-CTA tail: [0] FP64, [1] FP32 (nlev: none)
    size_t tail_smem[2] = {0, 0};     // its dynamic shared memory in bytes
    int tail_img[2] = {0, 0};         // elements of one sample's operator image of the tail levels
    double *timg64 = nullptr;         // the images, FP64 tail (every sample)
    float *timg32 = nullptr;          // FP32 tail
    double *Ainv = nullptr;           // coarsest inverse (FP64), nc x nc per sample
    double *M = nullptr;              // Gauss-Jordan work matrix [A | I], nc x 2nc per sample
    int *gj_status = nullptr;         // Gauss-Jordan status per sample (device)
    int *hstatus = nullptr;           // pinned host copy
    float *Ainv32 = nullptr;
    double *stage = nullptr;          // contiguous nx*ny*nz buffer for host transfers
    double *stage2 = nullptr;         // a second one, for transfers on the side stream
    cudaStream_t side = nullptr;      // overlaps host transfers with the iteration on the caller's stream
    dmg_ctx *twin = nullptr;          // dmg_solve_vjp's adjoint lane (twin_adjoint), created on first use
    cudaStream_t twin_s = nullptr;    // the stream the twin iterates on (lowest priority)
    cudaStream_t lead_s = nullptr;    // the forward solve of a two-lane pair (highest priority)
    cudaEvent_t ev_lead = nullptr;
    cudaEvent_t ev_twin = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_aux = nullptr;
    // dmg_solve_vjp_many (allocated on first use): two input staging buffers
    // (q then w, caller layout), two output staging buffers (u, qbar, Dbar,
    // mubar), an upload and a download stream, and their events
    double *mi_stage[2] = {nullptr, nullptr}, *mo_stage[2] = {nullptr, nullptr};
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_used[2] = {}, ev_ready_u[2] = {}, ev_ready[2] = {}, ev_out[2] = {};
    cudaEvent_t ev_in_q[2] = {}, ev_used_w[2] = {}, ev_qb[2] = {};   // two-lane stream of pairs
    bool many_ready = false;
    // pyramid pool (dmg_setup_pyramid): slot b's finest level is top_of[b]; level l
    // holds samples [0, L[l].g.nb), of which [top_first[l], top_first[l] + top_count[l])
    // have it as their finest level. Every other context is the case of one top
    // level (level 0, all samples).
    bool pyramid = false;
    int top_count[kMaxLevels] = {}, top_first[kMaxLevels] = {};
    std::vector<int> top_of;
    std::vector<long long> stage_off;   // per slot: its part of the contiguous staging buffers
    // per level: outputs of the slots whose finest level it is (U0l[0] = U0, ...)
    double *U0l[kMaxLevels] = {}, *T1l[kMaxLevels] = {}, *T2l[kMaxLevels] = {};
    double *U0 = nullptr;             // level-0 staging: user's u
    double *T1 = nullptr, *T2 = nullptr, *T3 = nullptr;  // level-0 staging: tangents / outputs
    double *partial = nullptr;        // reduction partials
    double *red = nullptr;            // reduction results (device, kRedSlots doubles per sample)
    double *hred = nullptr;           // pinned host copy of red (mapped: hred_d is its device address)
    double *hred_d = nullptr;
    int *hact_d = nullptr, *hact_a_d = nullptr;   // device addresses of the mapped hact, hact_a
    int *act = nullptr;               // device mask: sample still iterating
    const int *mask = nullptr;        // mask argument of the launches being issued: act, or NULL
                                      // while every sample iterates (no per-block mask load)
    int *hact = nullptr;              // pinned host copy of act
    // slot-level interface: per-slot state, the adjoint-phase mask, and one
    // step graph per direction ([0] forward and tangent phases, masked by act;
    // [1] adjoint phases, masked by act_a)
    std::vector<Slot> slots;
    // unrolled gradient: per-level work buffers and level-0 checkpoints (allocated on first use)
    ULevel un[kMaxLevels];
    bool un_ready = false;
    std::vector<double *> ck;
    int *act_a = nullptr, *hact_a = nullptr;
    Graph g_srv[2];
    bool step_open = false;
    std::vector<int> bcyc;            // per sample: cycles of the last call
    std::vector<double> brel;         // per sample: final relative residual of the last call
    dmgk::MixScalars *ms = nullptr;   // device scalars of the mixed-precision loop
    std::vector<void *> dev_allocs;
    size_t dev_bytes = 0;             // device memory held by the context
    unsigned long long launches = 0;
    char err[512] = {0};
    // CUDA graphs of the repeated steps, captured on first use on cap_stream:
    // [0] forward, [1] transposed; second index: [0] every sample active
    // (no mask), [1] masked by act (once some sample of a batch has converged)
    cudaStream_t cap_stream = nullptr;
    Graph g_mix[2][2], g_cyc[2][2], g_fix[2][2];
    // profiling: event pairs bracketing launches of one kernel on one level
    int prof_kernel = -1, prof_level = 0, prof_fp32 = 0;
    std::vector<cudaEvent_t> prof_ev;   // 2 per pair
    std::vector<int> prof_free;         // unused pairs
    std::vector<int> prof_direct;       // pairs recorded by direct launches since the last harvest
    std::vector<int> *prof_sink = nullptr;
    std::vector<int> prof_n;            // launches each pair brackets
    int prof_open = -1;                 // the pair of an open group of launches
    long long prof_count = 0;
    double prof_ms = 0.0;
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

// interior launch: block (32, 8), grid over interior x/y, blockIdx.z = sample * planes + plane
inline dim3 blk() { return dim3(32, 8, 1); }
// per-vertex kernels: blockIdx.x = 2 * (32-wide chunk of the half-row) + parity
inline dim3 grid_int(const Geom &g) {
    return dim3(2 * ((g.nhalf() + 31) / 32), (g.ny - 2 + 7) / 8, g.nb * (g.nz - 2));
}
// k_update / k_to_f32: elements m, m+1 of one half-row per thread; pairs
// 0 .. (nx - 2) / 4 cover the interior vertices of either parity
inline dim3 grid_int_pair(const Geom &g) {
    return dim3(2 * (((g.nx - 2) / 4 + 1 + 31) / 32), (g.ny - 2 + 7) / 8, g.nz == 1 ? g.nb : g.nb * (g.nz - 2));
}
inline dim3 grid_all(const Geom &g) { return dim3(2 * ((g.nhalf() + 31) / 32), (g.ny + 7) / 8, g.nb * g.nz); }
// half-sweeps: x covers the (nx-1)/2 vertices of one colour in a row
inline dim3 grid_half(const Geom &g) {
    return dim3(((g.nx - 1) / 2 + 31) / 32, (g.ny - 2 + 7) / 8, g.nb * (g.nz - 2));
}
// 2D levels (nz == 1): blockIdx.z = sample
inline dim3 grid_half2(const Geom &g) { return dim3(((g.nx - 1) / 2 + 31) / 32, (g.ny - 2 + 7) / 8, g.nb); }
inline dim3 grid_int2(const Geom &g) { return dim3(2 * ((g.nhalf() + 31) / 32), (g.ny - 2 + 7) / 8, g.nb); }
inline dim3 grid_all2(const Geom &g) { return dim3(2 * ((g.nhalf() + 31) / 32), (g.ny + 7) / 8, g.nb); }

// dmg_debug_grad_per_vertex: the per-vertex gradient kernels for both face means
std::atomic<int> g_grad_per_vertex{0};

// Dbar and mubar of <w, u> from u and lam on a 3D level, in the level's
// layout: the tiled kernel for the arithmetic face mean (bitwise k_grad, fewer
// FP64 operations), k_grad for the harmonic one. dnat / mnat: that output is
// written in the natural layout (tiled kernel only: callers ask for it where
// grad_tiled() held, and the tiled kernel then runs whatever the hook says by
// now).
inline bool grad_tiled(bool harm) { return !harm && !g_grad_per_vertex.load(); }

inline void launch_grad(cudaStream_t s, const Geom &g, const double *u, const double *lam, const double *D,
                        double ih2, bool harm, double *Dbar, double *mubar, bool dnat = false, bool mnat = false) {
    if (!dnat && !mnat && !grad_tiled(harm)) {
        dmgk::k_grad<<<grid_all(g), blk(), 0, s>>>(g, u, lam, D, ih2, harm, Dbar, mubar);
        return;
    }
    const int nzb = (g.nz + dmgk::kGradTZ - 1) / dmgk::kGradTZ;
    const dim3 grid((g.nx + dmgk::kGradTX - 1) / dmgk::kGradTX, (g.ny + dmgk::kGradTY - 1) / dmgk::kGradTY,
                    g.nb * nzb);
    dmgk::k_grad_am<<<grid, dim3(dmgk::kGradTX, dmgk::kGradTY, dmgk::kGradTZ), 0, s>>>(g, u, lam, nzb, ih2, Dbar,
                                                                                          dnat, mubar, mnat);
}

// the same on a 2D level (k_grad2_am / k_grad2)
inline void launch_grad2(cudaStream_t s, const Geom &g, const double *u, const double *lam, const double *D,
                         double ih2, bool harm, double *Dbar, double *mubar, bool dnat = false, bool mnat = false) {
    if (!dnat && !mnat && !grad_tiled(harm)) {
        dmgk::k_grad2<<<grid_all2(g), blk(), 0, s>>>(g, u, lam, D, ih2, harm, Dbar, mubar);
        return;
    }
    const dim3 grid((g.nx + dmgk::kGrad2TX - 1) / dmgk::kGrad2TX, (g.ny + dmgk::kGrad2TY - 1) / dmgk::kGrad2TY, g.nb);
    dmgk::k_grad2_am<<<grid, dim3(dmgk::kGrad2TX, dmgk::kGrad2TY), 0, s>>>(g, u, lam, ih2, Dbar, dnat, mubar, mnat);
}
// the same with a tuned block shape b (b.x threads along the half-row, b.y rows)
inline dim3 grid_half(const Geom &g, dim3 b) {
    return dim3(((g.nx - 1) / 2 + b.x - 1) / b.x, (g.ny - 2 + b.y - 1) / b.y, g.nb * (g.nz - 2));
}
// the FP32 pair kernels (k_smooth_half32, k_residual_colour32,
// k_prolong_smooth32): one thread per
// two elements m, m+1 of a half-row; interior vertices i = 2m + parity <= nx - 2
// have m <= (nx - 2) / 2, so pairs 0 .. (nx - 2) / 4 cover them
inline dim3 grid_pair(const Geom &g, dim3 b) {
    const int pairs = (g.nx - 2) / 4 + 1;
    return dim3((pairs + b.x - 1) / b.x, (g.ny - 2 + b.y - 1) / b.y, g.nb * (g.nz - 2));
}

dmg_status check_launch(dmg_ctx *c, const char *what) {
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, DMG_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return DMG_OK;
}

// Launch with programmatic stream serialization: the kernel may be scheduled
// while its predecessor in the stream drains, and waits for it in pdl_wait()
// before its first read (every kernel launched this way calls it first).
template <class... P, class... A>
dmg_status launch_pdl(dmg_ctx *c, const char *what, void (*k)(P...), dim3 grid, dim3 block, size_t smem,
                      cudaStream_t s, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    c->launches++;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DMG_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    }
    return DMG_OK;
}

// Host-side fault injection for tests: when > 0, the allocation with this
// ordinal (counting from the next one, process-wide) fails as if the device
// were out of memory.
std::atomic<long long> g_fail_alloc_at{0};

template <class T>
dmg_status dalloc(dmg_ctx *c, T **p, size_t n) {
    void *q = nullptr;
    const long long k = g_fail_alloc_at.load();
    if (k > 0 && g_fail_alloc_at.fetch_sub(1) == 1)
        return fail(c, DMG_ENOMEM, "cudaMalloc of %zu bytes failed: injected allocation failure", n * sizeof(T));
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DMG_ENOMEM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T),
                    cudaGetErrorString(e));
    }
    c->dev_allocs.push_back(q);
    c->dev_bytes += n * sizeof(T);
    *p = static_cast<T *>(q);
    return DMG_OK;
}

// --- profiling hooks -------------------------------------------------------
// A ProfScope brackets the launches of one kernel (kind, level, precision)
// with an event pair; in a graph capture the records become event nodes that
// every replay re-records, and the pair is harvested after each replay.
// Brackets launches of the profiled kernel with an event pair. A group scope
// (around a run of consecutive launches of the kernel, such as the half-sweeps
// of smooth()) brackets the whole run with one pair, and the scopes of the
// launches inside it only count them: per-launch event nodes cost a few
// microseconds each, which a run of n launches spreads over n.
struct ProfScope {
    dmg_ctx *c;
    cudaStream_t s;
    int idx = -1;
    bool group = false;
    ProfScope(dmg_ctx *c_, int kernel, int level, int fp32, cudaStream_t s_, bool group_ = false) : c(c_), s(s_) {
        if (c->prof_kernel == kernel && c->prof_level == level && c->prof_fp32 == fp32) {
            if (c->prof_open >= 0) {
                c->prof_n[c->prof_open]++;   // inside an open group
                return;
            }
            if (c->prof_free.empty()) return;
            idx = c->prof_free.back();
            c->prof_free.pop_back();
            c->prof_n[idx] = group_ ? 0 : 1;
            if (group_) {
                group = true;
                c->prof_open = idx;
            }
            record(c->prof_ev[2 * idx]);
        }
    }
    // an event node inside a capture (prof_sink set), a plain record outside
    void record(cudaEvent_t e) const {
        if (c->prof_sink) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
        else cudaEventRecord(e, s);
    }
    ~ProfScope() {
        if (idx >= 0) {
            if (group) c->prof_open = -1;
            record(c->prof_ev[2 * idx + 1]);
            (c->prof_sink ? c->prof_sink : &c->prof_direct)->push_back(idx);
        }
    }
};

// add the durations of completed pairs; release them unless a graph owns them
void prof_harvest(dmg_ctx *c, std::vector<int> &pairs, bool release) {
    for (int idx : pairs) {
        float ms = 0.f;
        if (c->prof_n[idx] > 0 &&
            cudaEventElapsedTime(&ms, c->prof_ev[2 * idx], c->prof_ev[2 * idx + 1]) == cudaSuccess) {
            c->prof_ms += ms;
            c->prof_count += c->prof_n[idx];
        } else {
            cudaGetLastError();
        }
        if (release) c->prof_free.push_back(idx);
    }
    if (release) pairs.clear();
}

void graphs_reset(dmg_ctx *c) {
    for (Graph *set : {&c->g_mix[0][0], &c->g_cyc[0][0], &c->g_fix[0][0]})
        for (int t = 0; t < 4; t++) {
            if (set[t].exec) cudaGraphExecDestroy(set[t].exec);
            for (int idx : set[t].prof) c->prof_free.push_back(idx);
            set[t] = Graph();
        }
    for (Graph &G : c->g_srv) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        for (int idx : G.prof) c->prof_free.push_back(idx);
        G = Graph();
    }
}

// dst = src, n elements, by a kernel on stream s (double2 when both are 16-byte
// aligned and n is even)
template <class T>
dmg_status dcopy(dmg_ctx *c, T *dst, const T *src, size_t n, cudaStream_t s) {
    if (n == 0) return DMG_OK;
    const int blocks = 148 * 8;
    if (sizeof(T) == 8 && n % 2 == 0 && ((uintptr_t)dst % 16) == 0 && ((uintptr_t)src % 16) == 0)
        dmgk::k_copy<double2><<<blocks, 256, 0, s>>>(reinterpret_cast<const double2 *>(src),
                                                     reinterpret_cast<double2 *>(dst), (long long)(n / 2));
    else
        dmgk::k_copy<T><<<blocks, 256, 0, s>>>(src, dst, (long long)n);
    return check_launch(c, "copy");
}

// --- staging between the caller's contiguous arrays and the split layout -------
// Device (or managed) caller arrays are read/written in place by the gather and
// scatter kernels; host arrays go through the contiguous staging buffer.
bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// gather/scatter grid: x over the vertices of one sample, y over samples
// k_gather / k_scatter: four consecutive vertices of a row per thread, blk() blocks
inline dim3 quad_grid(const Geom &g) {
    return dim3(((g.nx + 3) / 4 + 31) / 32, (g.ny + 7) / 8, g.nb * g.nz);
}

// level-0 geometry of every sample (slot < 0), or the geometry of one slot's
// finest level (a single sample)
inline Geom geom0(const dmg_ctx *c, int slot) {
    if (slot < 0) return c->L[0].g;
    Geom g = c->L[c->top_of[slot]].g;
    g.nb = 1;
    return g;
}

// src (caller layout, every sample or one slot's sample) -> dst (split layout of
// the same samples; dst already points at the slot's part)
dmg_status stage_in(dmg_ctx *c, const double *src, double *dst, bool zero_boundary, cudaStream_t s, int slot = -1,
                    double *buf = nullptr) {
    const Geom g = geom0(c, slot);
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t bytes = n * g.nb * sizeof(double);
    const double *from = src;
    if (!is_device_ptr(src)) {
        double *st = (buf ? buf : c->stage) + (slot < 0 ? 0 : c->stage_off[slot]);
        CUDA_TRY(c, cudaMemcpyAsync(st, src, bytes, cudaMemcpyHostToDevice, s));
        from = st;
    }
    dmgk::k_gather<<<quad_grid(g), blk(), 0, s>>>(g, from, dst, zero_boundary ? 1 : 0);
    return check_launch(c, "gather");
}

dmg_status stage_out(dmg_ctx *c, const double *src, double *dst, cudaStream_t s, int slot = -1,
                     double *buf = nullptr) {
    const Geom g = geom0(c, slot);
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t bytes = n * g.nb * sizeof(double);
    if (is_device_ptr(dst)) {
        dmgk::k_scatter<<<quad_grid(g), blk(), 0, s>>>(g, src, dst);
        return check_launch(c, "scatter");
    }
    double *st = (buf ? buf : c->stage) + (slot < 0 ? 0 : c->stage_off[slot]);
    dmgk::k_scatter<<<quad_grid(g), blk(), 0, s>>>(g, src, st);
    TRY(check_launch(c, "scatter"));
    CUDA_TRY(c, cudaMemcpyAsync(dst, st, bytes, cudaMemcpyDeviceToHost, s));
    return DMG_OK;
}

// Dbar and mubar of <w, u> from level-0 u and lam into the caller's arrays
// (either may be NULL): an array on the device is written directly by the
// tiled kernels (arithmetic face mean), any other through T1 / T2 and
// stage_out.
dmg_status grad_out(dmg_ctx *c, const double *u, const double *lam, double *Dbar, double *mubar, cudaStream_t s) {
    const Level &l = c->L[0];
    const double ih2 = 1.0 / (l.h * l.h);
    const bool harm = c->p.face_mean == DMG_FACE_HARMONIC;
    const bool tiled = grad_tiled(harm);
    const bool dnat = tiled && Dbar && is_device_ptr(Dbar), mnat = tiled && mubar && is_device_ptr(mubar);
    double *Dt = Dbar ? (dnat ? Dbar : c->T1) : nullptr, *mt = mubar ? (mnat ? mubar : c->T2) : nullptr;
    {
        ProfScope ps(c, DMG_KERNEL_GRAD, 0, 0, s);
        if (c->dim == 2)
            launch_grad2(s, l.g, u, lam, l.D, ih2, harm, Dt, mt, dnat, mnat);
        else
            launch_grad(s, l.g, u, lam, l.D, ih2, harm, Dt, mt, dnat, mnat);
        TRY(check_launch(c, "grad"));
    }
    if (Dbar && !dnat) TRY(stage_out(c, c->T1, Dbar, s));
    if (mubar && !mnat) TRY(stage_out(c, c->T2, mubar, s));
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

// one RB-GS half-sweep of `color` on level lev
template <class T>
dmg_status half_sweep(dmg_ctx *c, int lev, int color, cudaStream_t s) {
    Level &l = c->L[lev];
    ProfScope ps(c, DMG_KERNEL_SMOOTH, lev, sizeof(T) == 4, s);
    if (c->dim == 2) {
        return dispatch<T>(c, l, [&](auto cf) {
            if constexpr (sizeof(T) == 4) {
                constexpr bool H = decltype(cf)::harmonic;
                const dim3 b = blk();
                const dim3 gr(((l.g.nx - 2) / 4 + 1 + b.x - 1) / b.x, (l.g.ny - 2 + b.y - 1) / b.y, l.g.nb);
                return launch_pdl(c, "smooth", dmgk::k_smooth_half2_pair32<H>, gr, b, 0, s, l.g, l.u32,
                                  (const float *)l.f32, cf, color, (const int *)c->mask);
            } else {
                return launch_pdl(c, "smooth", dmgk::k_smooth_half2<T, decltype(cf)>, grid_half2(l.g), blk(), 0, s,
                                  l.g, U<T>(l), (const T *)F<T>(l), cf, color, (const int *)c->mask);
            }
        });
    }
    if constexpr (sizeof(T) == 4) {
        return with_coef32(c, l, [&](auto cf) {
            constexpr bool H = decltype(cf)::harmonic;
            const dim3 b = c->tb[1][lev];
            if (c->nb == 1)
                return launch_pdl(c, "smooth", dmgk::k_smooth_half32<H, false>, grid_pair(l.g, b), b, 0, s, l.g,
                                  l.u32, (const float *)l.f32, cf, color, (const int *)nullptr);
            return launch_pdl(c, "smooth", dmgk::k_smooth_half32<H, true>, grid_pair(l.g, b), b, 0, s, l.g, l.u32,
                              (const float *)l.f32, cf, color, (const int *)c->mask);
        });
    } else {
        const dim3 b = c->tb[0][lev];
        return launch_pdl(c, "smooth", dmgk::k_smooth_half<T, dmgk::FaceCoef<T>>, grid_half(l.g, b), b, 0, s, l.g,
                          U<T>(l), (const T *)F<T>(l), coef64(l), color, (const int *)c->mask);
    }
}

// nsweeps RB-GS sweeps; each sweep is the half-sweep of colour `first` then the other
template <class T>
dmg_status smooth(dmg_ctx *c, int lev, int first, int nsweeps, cudaStream_t s) {
    ProfScope ps(c, DMG_KERNEL_SMOOTH, lev, sizeof(T) == 4, s, true);
    for (int it = 0; it < nsweeps; it++) {
        TRY(half_sweep<T>(c, lev, first, s));
        TRY(half_sweep<T>(c, lev, 1 - first, s));
    }
    return DMG_OK;
}

// f_{l+1} = R (f_l - A_l u_l), u_{l+1} = 0 (the restriction kernels write
// both). zero_colour >= 0: the defect
// vanishes on that colour (the last half-sweep updated it), so it is formed on
// the other colour only and the restriction reads only that colour.
// the coarse level lev+1 seen with the samples of level lev only (a pyramid's
// coarse levels also hold the samples whose finest level they are; transfers
// between lev and lev+1 touch the samples of lev)
inline Level coarse_of(const dmg_ctx *c, int lev) {
    Level v = c->L[lev + 1];
    v.g.nb = c->L[lev].g.nb;
    return v;
}

template <class T>
dmg_status restrict_defect(dmg_ctx *c, int lev, int zero_colour, cudaStream_t s) {
    Level &l = c->L[lev];
    Level cl = coarse_of(c, lev);
    ProfScope ps(c, DMG_KERNEL_RESTRICT, lev, sizeof(T) == 4, s);
    if (c->dim == 2 && zero_colour >= 0) {
        // the defect on one colour and its 9-point full weighting
        const int nz = 1 - zero_colour;
        TRY(dispatch<T>(c, l, [&](auto cf) {
            return launch_pdl(c, "residual_colour", dmgk::k_residual_colour2<T, decltype(cf)>, grid_half2(l.g), blk(),
                              0, s, l.g, (const T *)U<T>(l), (const T *)F<T>(l), cf, R<T>(l), nz,
                              (const int *)c->mask);
        }));
        if (nz == 0)
            return launch_pdl(c, "restrict_colour", dmgk::k_restrict_colour2<T, 0>, grid_int2(cl.g), blk(), 0, s, l.g,
                              (const T *)R<T>(l), cl.g, F<T>(cl), U<T>(cl), (const int *)c->mask);
        return launch_pdl(c, "restrict_colour", dmgk::k_restrict_colour2<T, 1>, grid_int2(cl.g), blk(), 0, s, l.g,
                          (const T *)R<T>(l), cl.g, F<T>(cl), U<T>(cl), (const int *)c->mask);
    }
    if (c->dim == 2) {   // full defect and 9-point full weighting
        TRY(dispatch<T>(c, l, [&](auto cf) {
            dmgk::k_residual2<T><<<grid_int2(l.g), blk(), 0, s>>>(l.g, U<T>(l), F<T>(l), cf, R<T>(l), c->mask);
            return check_launch(c, "residual");
        }));
        dmgk::k_restrict2<T><<<grid_int2(cl.g), blk(), 0, s>>>(l.g, R<T>(l), cl.g, F<T>(cl), U<T>(cl), c->mask);
        return check_launch(c, "restrict");
    }
    if (zero_colour >= 0) {
        const int nz = 1 - zero_colour;   // colour carrying the defect
        if constexpr (sizeof(T) == 4) {
            TRY(with_coef32(c, l, [&](auto cf) {
                constexpr bool H = decltype(cf)::harmonic;
                const dim3 b = c->tb[1][lev];
                if (c->nb == 1)
                    return launch_pdl(c, "residual_colour", dmgk::k_residual_colour32<H, false>, grid_pair(l.g, b), b,
                                      0, s, l.g, (const float *)l.u32, (const float *)l.f32, cf, l.r32, nz,
                                      (const int *)nullptr);
                return launch_pdl(c, "residual_colour", dmgk::k_residual_colour32<H, true>, grid_pair(l.g, b), b, 0,
                                  s, l.g, (const float *)l.u32, (const float *)l.f32, cf, l.r32, nz,
                                  (const int *)c->mask);
            }));
        } else {
            const dim3 b = c->tb[0][lev];
            TRY(launch_pdl(c, "residual_colour", dmgk::k_residual_colour<T, dmgk::FaceCoef<T>>, grid_half(l.g, b), b,
                           0, s, l.g, (const T *)U<T>(l), (const T *)F<T>(l), coef64(l), R<T>(l), nz,
                           (const int *)c->mask));
        }
        // fine vertex 2I+offset has colour parity(offset); the defect lives on colour nz
        if (nz == 0)
            TRY(launch_pdl(c, "restrict_colour", dmgk::k_restrict_colour<T, 0>, grid_int(cl.g), blk(), 0, s, l.g,
                           (const T *)R<T>(l), cl.g, F<T>(cl), U<T>(cl), (const int *)c->mask));
        else
            TRY(launch_pdl(c, "restrict_colour", dmgk::k_restrict_colour<T, 1>, grid_int(cl.g), blk(), 0, s, l.g,
                           (const T *)R<T>(l), cl.g, F<T>(cl), U<T>(cl), (const int *)c->mask));
    } else {
        TRY(dispatch<T>(c, l, [&](auto cf) {
            dmgk::k_residual<T><<<grid_int(l.g), blk(), 0, s>>>(l.g, U<T>(l), F<T>(l), cf, R<T>(l), c->mask);
            return check_launch(c, "residual");
        }));
        dmgk::k_restrict<T><<<grid_int(cl.g), blk(), 0, s>>>(l.g, R<T>(l), cl.g, F<T>(cl), U<T>(cl), c->mask);
        TRY(check_launch(c, "restrict"));
    }
    return DMG_OK;
}

// levels of at least this many vertices (all samples) take the correction on
// one colour and plain half-sweeps instead of the fused launch
constexpr long long kSplitProlongVertices = 1LL << 22;

inline bool split_prolong_level(const Level &l) { return (long long)l.g.sb * l.g.nb >= kSplitProlongVertices; }

// u_lev += P u_{lev+1} on the vertices of `color` only (k_prolong_colour32):
// the values the half-sweep of the other colour, which must follow, reads.
dmg_status prolong_colour32(dmg_ctx *c, int lev, int color, cudaStream_t s) {
    Level &l = c->L[lev];
    Level cl = coarse_of(c, lev);
    ProfScope ps(c, DMG_KERNEL_PROLONG, lev, 1, s);
    const dim3 b = c->tb[1][lev];
    if (c->nb == 1)
        return launch_pdl(c, "prolong_colour", dmgk::k_prolong_colour32<false>, grid_pair(l.g, b), b, 0, s, l.g,
                          l.u32, cl.g, (const float *)cl.u32, color, (const int *)nullptr);
    return launch_pdl(c, "prolong_colour", dmgk::k_prolong_colour32<true>, grid_pair(l.g, b), b, 0, s, l.g, l.u32,
                      cl.g, (const float *)cl.u32, color, (const int *)c->mask);
}

// u_lev += P u_{lev+1}, then the half-sweep of colour `color` on lev, in one
// FP32 launch that stores only the colour's new values (k_prolong_smooth32):
// only the other colour's corrected values are ever read (by this half-sweep),
// so they are formed on the fly. The half-sweep of the other colour must follow.
dmg_status prolong_smooth32(dmg_ctx *c, int lev, int color, cudaStream_t s) {
    Level &l = c->L[lev];
    Level cl = coarse_of(c, lev);
    ProfScope ps(c, DMG_KERNEL_PROLONG, lev, 1, s);
    return with_coef32(c, l, [&](auto cf) {
        constexpr bool H = decltype(cf)::harmonic;
        const dim3 b = c->tb[1][lev];
        if (c->nb == 1)
            return launch_pdl(c, "prolong_smooth", dmgk::k_prolong_smooth32<H, false>, grid_pair(l.g, b), b, 0, s,
                              l.g, l.u32, (const float *)l.f32, cf, cl.g, (const float *)cl.u32, color,
                              (const int *)nullptr);
        return launch_pdl(c, "prolong_smooth", dmgk::k_prolong_smooth32<H, true>, grid_pair(l.g, b), b, 0, s, l.g,
                          l.u32, (const float *)l.f32, cf, cl.g, (const float *)cl.u32, color, (const int *)c->mask);
    });
}

template <class T>
dmg_status prolong(dmg_ctx *c, int lev, cudaStream_t s) {
    Level &l = c->L[lev];
    Level cl = coarse_of(c, lev);
    ProfScope ps(c, DMG_KERNEL_PROLONG, lev, sizeof(T) == 4, s);
    if (c->dim == 2) {
        dim3 grid((cl.g.nx - 1 + 31) / 32, (cl.g.ny - 1 + 7) / 8, l.g.nb);   // coarse cells
        return launch_pdl(c, "prolong", dmgk::k_prolong_add2<T>, grid, blk(), 0, s, cl.g, (const T *)U<T>(cl), l.g,
                          U<T>(l), (const int *)c->mask);
    }
    dim3 grid((cl.g.nx - 1 + 31) / 32, (cl.g.ny - 1 + 7) / 8, l.g.nb * (cl.g.nz - 1));   // coarse cells
    return launch_pdl(c, "prolong", dmgk::k_prolong_add<T>, grid, blk(), 0, s, cl.g, (const T *)U<T>(cl), l.g,
                      U<T>(l), (const int *)c->mask);
}


// per-level coefficient object of the type a kernel instantiation expects
inline dmgk::FaceCoef<double> make_coef(const Level &l, dmgk::FaceCoef<double>) { return coef64(l); }
template <bool H>
inline dmgk::VertCoef<float, H> make_coef(const Level &l, dmgk::VertCoef<float, H>) {
    return dmgk::VertCoef<float, H>{l.Dh32, l.mu32};
}

template <class T>
T *tail_image(dmg_ctx *c);
template <>
double *tail_image<double>(dmg_ctx *c) { return c->timg64; }
template <>
float *tail_image<float>(dmg_ctx *c) { return c->timg32; }

// the arguments of the tail kernels of precision T (levels tail_first .. nlev-1)
template <class T, class C>
void tail_args(dmg_ctx *c, C cf0, dmgk::TailArgs<T, C> &a) {
    const int t = sizeof(T) == 4;
    const int l0 = c->tail_first[t];
    a.nl = c->nlev - l0;
    for (int l = 0; l < a.nl; l++) {
        Level &lv = c->L[l0 + l];
        a.L[l].g = lv.g;
        a.L[l].gs = smem_geom(lv.g);
        a.L[l].u = U<T>(lv);
        a.L[l].f = F<T>(lv);
        a.L[l].c = make_coef(lv, cf0);
        a.L[l].dv = tail_div(lv.g);
    }
    a.img = tail_image<T>(c);
    a.img_elems = c->tail_img[t];
    a.Ainv = AINV<T>(c);
    a.nc = c->nc;
    a.act = c->mask;
}

// the operator images of the tail levels of samples first .. first+count-1
// (after their coefficients are built)
template <class T>
dmg_status build_tail_image(dmg_ctx *c, int first, int count, cudaStream_t s) {
    const int t = sizeof(T) == 4;
    if (c->tail_first[t] >= c->nlev || !tail_image<T>(c)) return DMG_OK;
    return dispatch<T>(c, c->L[c->tail_first[t]], [&](auto cf0) -> dmg_status {
        using C = decltype(cf0);
        dmgk::TailArgs<T, C> a{};
        tail_args<T>(c, cf0, a);
        dmgk::k_tail_image<T, C><<<count, 1024, 0, s>>>(a, tail_image<T>(c), first);
        return check_launch(c, "tail_image");
    });
}

// The levels tail_first .. nlev-1 of one V-cycle (descent, exact coarsest
// solve, ascent) in a launch of one block per sample working in shared memory.
template <class T>
dmg_status launch_tail(dmg_ctx *c, int npre, int npost, int pre_first, int post_first, cudaStream_t s) {
    const int t = sizeof(T) == 4;
    const int l0 = c->tail_first[t];
    ProfScope ps(c, DMG_KERNEL_TAIL, l0, t, s);
    return dispatch<T>(c, c->L[l0], [&](auto cf0) -> dmg_status {
        using C = decltype(cf0);
        dmgk::TailArgs<T, C> a{};
        tail_args<T>(c, cf0, a);
        a.npre = npre;
        a.npost = npost;
        a.pre_first = pre_first;
        a.post_first = post_first;
        a.load_u = l0 == 0;   // the V-cycle of the finest level continues from the current iterate
        return launch_pdl(c, "vcycle_tail", dmgk::k_vcycle_tail<T, C>, dim3(c->nb), dim3(1024), c->tail_smem[t], s,
                          a);
    });
}

// exact coarsest solve by one grid launch (used when the tail does not fit in
// shared memory)
template <class T>
dmg_status coarse_solve(dmg_ctx *c, cudaStream_t s) {
    Level &l = c->L[c->nlev - 1];
    int threads = c->nc < 32 ? 32 : (c->nc > 512 ? 512 : ((c->nc + 31) / 32) * 32);
    if (c->dim == 2)
        dmgk::k_coarse_solve2<T><<<c->nb, threads, c->nc * sizeof(T), s>>>(l.g, AINV<T>(c), c->nc, F<T>(l), U<T>(l),
                                                                            c->mask);
    else
        dmgk::k_coarse_solve<T><<<c->nb, threads, c->nc * sizeof(T), s>>>(l.g, AINV<T>(c), c->nc, F<T>(l), U<T>(l),
                                                                           c->mask);
    return check_launch(c, "coarse_solve");
}

// One V-cycle at level lev on (u_lev, f_lev), in place (Sec. 2.2, Fig. 1 left).
// transposed: the V-cycle whose preconditioner is the transpose of the forward
// one (Sec. 2.4): nu2 pre-sweeps and nu1 post-sweeps, colour orders reversed.
template <class T>
dmg_status vcycle(dmg_ctx *c, int lev, bool transposed, cudaStream_t s) {
    int post_first = c->p.symmetric ? 1 : 0;
    int npre = transposed ? c->p.nu2 : c->p.nu1, npost = transposed ? c->p.nu1 : c->p.nu2;
    int pre_first = transposed ? 1 - post_first : 0;
    int postf = transposed ? 1 : post_first;
    if (lev == c->tail_first[sizeof(T) == 4]) return launch_tail<T>(c, npre, npost, pre_first, postf, s);
    if (lev == c->nlev - 1) return coarse_solve<T>(c, s);
    TRY(smooth<T>(c, lev, pre_first, npre, s));
    // after pre-smoothing the defect is zero on the colour updated last
    TRY(restrict_defect<T>(c, lev, npre > 0 ? 1 - pre_first : -1, s));
    TRY(vcycle<T>(c, lev + 1, transposed, s));
    if (c->dim == 2 && npost > 0 && !c->p.split_prolong) {
        // the correction on the colour the first post half-sweep reads
        Level &l = c->L[lev];
        Level cl = coarse_of(c, lev);
        {
            ProfScope ps(c, DMG_KERNEL_PROLONG, lev, sizeof(T) == 4, s);
            TRY(launch_pdl(c, "prolong_colour", dmgk::k_prolong_colour2<T>, grid_half2(l.g), blk(), 0, s, cl.g,
                           (const T *)U<T>(cl), l.g, U<T>(l), 1 - postf, (const int *)c->mask));
        }
        return smooth<T>(c, lev, postf, npost, s);
    }
    if (sizeof(T) == 4 && c->dim == 3 && npost > 0 && !c->p.split_prolong) {
        if (split_prolong_level(c->L[lev])) {
            // the correction on the colour the first post half-sweep reads
            TRY(prolong_colour32(c, lev, 1 - postf, s));
            return smooth<T>(c, lev, postf, npost, s);
        }
        // correction fused into the first post half-sweep; its other half next
        TRY(prolong_smooth32(c, lev, postf, s));
        TRY(half_sweep<T>(c, lev, 1 - postf, s));
        return smooth<T>(c, lev, postf, npost - 1, s);
    }
    TRY(prolong<T>(c, lev, s));
    TRY(smooth<T>(c, lev, postf, npost, s));
    return DMG_OK;
}

// --- reductions ------------------------------------------------------------------
constexpr int kSlots = dmgk::kRedSlots;

// copy the reduction slots of every sample to pinned host memory (a kernel
// writing through the mapping: no copy engine, so a step's read-back never
// queues behind bulk host transfers on other streams)
dmg_status enqueue_readback(dmg_ctx *c, cudaStream_t s) {
    return dcopy(c, c->hred_d, c->red, (size_t)kSlots * c->nb, s);
}

// wait for the stream; the results are in hred[sample * kSlots + slot]
dmg_status sync_read(dmg_ctx *c, cudaStream_t s) {
    CUDA_TRY(c, cudaStreamSynchronize(s));
    prof_harvest(c, c->prof_direct, true);
    return DMG_OK;
}

inline double hred(const dmg_ctx *c, int smp, int slot) { return c->hred[smp * kSlots + slot]; }

// the host mask to the device (the next launches see it; a replayed graph
// reads it at run time)
dmg_status push_act(dmg_ctx *c, cudaStream_t s) {
    return dcopy(c, c->act, (const int *)c->hact_d, (size_t)c->nb, s);
}

// end of an API call: wait for the stream, harvest direct profiling pairs
dmg_status end_call(dmg_ctx *c, cudaStream_t s) {
    CUDA_TRY(c, cudaStreamSynchronize(s));
    prof_harvest(c, c->prof_direct, true);
    return DMG_OK;
}

dmg_status finish_reduce(dmg_ctx *c, cudaStream_t s) {
    TRY(enqueue_readback(c, s));
    return sync_read(c, s);
}

// ||x||_2^2 over interior of each sample of a level-0 FP64 array -> red[sample][slot]
dmg_status norm2_async(dmg_ctx *c, const double *x, int slot, cudaStream_t s) {
    if (c->dim == 2)
        dmgk::k_norm2_2d<<<dim3(kNormBlocks, c->nb), 256, 0, s>>>(c->L[0].g, x, c->partial);
    else
        dmgk::k_norm2<<<dim3(kNormBlocks, c->nb), 256, 0, s>>>(c->L[0].g, x, c->partial);
    TRY(check_launch(c, "norm2"));
    dmgk::k_reduce_final<<<c->nb, 256, 0, s>>>(c->partial, kNormBlocks, c->red, slot, nullptr);
    return check_launch(c, "reduce");
}

// ||f - A u||^2 (FP64, level 0) of each active sample -> red[sample][slot];
// with r32: the FP32 right-hand side r * 2^-e_prev
dmg_status resid_norm_async(dmg_ctx *c, const double *u, const double *f, float *r32, int slot, const int *act,
                            cudaStream_t s) {
    Level &l = c->L[0];
    {
        ProfScope ps(c, DMG_KERNEL_RESIDUAL, 0, 0, s);
        if (c->dim == 2)
            dmgk::k_resid_norm2<double><<<dim3(kNormBlocks, c->nb), 256, 0, s>>>(l.g, u, f, coef64(l), r32, c->ms,
                                                                                 c->partial, act);
        else
            dmgk::k_resid_norm<double><<<dim3(kNormBlocks, c->nb), 256, 0, s>>>(l.g, u, f, coef64(l),
                                                                                (double *)nullptr, r32, c->ms,
                                                                                c->partial, act);
        TRY(check_launch(c, "resid_norm"));
    }
    dmgk::k_reduce_final<<<c->nb, 256, 0, s>>>(c->partial, kNormBlocks, c->red, slot, act);
    return check_launch(c, "reduce");
}

// --- CUDA graphs ---------------------------------------------------------------------
// Capture body(stream) once on the context's capture stream; kernels launched
// while capturing are counted per replay instead of as launches.
template <class Body>
dmg_status capture(dmg_ctx *c, Graph &G, Body body) {
    if (G.exec) return DMG_OK;
    cudaStream_t cs = c->cap_stream;
    unsigned long long l0 = c->launches;
    std::vector<int> *saved = c->prof_sink;
    c->prof_sink = &G.prof;
    CUDA_TRY(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    dmg_status st = body(cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    c->prof_sink = saved;
    G.launches = c->launches - l0;
    c->launches = l0;
    if (st != DMG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(c, DMG_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&G.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        G.exec = nullptr;
        return fail(c, DMG_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
    }
    return DMG_OK;
}

dmg_status replay(dmg_ctx *c, Graph &G, cudaStream_t s) {
    CUDA_TRY(c, cudaGraphLaunch(G.exec, s));
    c->launches += G.launches;
    return DMG_OK;
}

void info_reset(dmg_info *info) {
    if (!info) return;
    memset(info, 0, sizeof(*info));
}

// --- per-sample convergence -----------------------------------------------------------
// Every sample of a batch iterates until its own relative residual meets rtol;
// a sample that has converged is switched off in the device mask, so its
// iterate is not touched again and it ends with exactly the cycles it would
// run alone. Samples with a zero right-hand side start converged (u = 0).
struct Progress {
    std::vector<double> nf;   // ||f_s||
    int active = 0;
};

// after the norms of the right-hand sides are in hred slot 0: set up the mask
dmg_status progress_start(dmg_ctx *c, Progress &P, dmg_info *info, cudaStream_t s) {
    c->bcyc.assign(c->nb, 0);
    c->brel.assign(c->nb, 0.0);
    P.nf.assign(c->nb, 0.0);
    P.active = 0;
    for (int b = 0; b < c->nb; b++) {
        const double n2 = hred(c, b, 0);
        if (!std::isfinite(n2)) {
            if (c->nb == 1) return fail(c, DMG_ENAN, "right-hand side is not finite");
            return fail(c, DMG_ENAN, "right-hand side of sample %d is not finite", b);
        }
        P.nf[b] = std::sqrt(n2);
        c->hact[b] = P.nf[b] > 0.0;
        if (c->hact[b]) {
            c->brel[b] = 1.0;
            P.active++;
        }
    }
    if (info) { info->cycles = 0; info->outer = 0; info->rel_residual = 0.0; }
    return P.active ? push_act(c, s) : DMG_OK;
}

// after step `step` (cycles = cycles of one step) with the residual norms in
// hred slot 0: record, retire converged samples; done = every sample has
// converged (or the tolerance is not used: fixed)
dmg_status progress_step(dmg_ctx *c, Progress &P, int step, int cycles, bool fixed, dmg_info *info, bool &done,
                         cudaStream_t s) {
    double worst = 0.0;
    bool changed = false;
    for (int b = 0; b < c->nb; b++) {
        if (!c->hact[b]) continue;
        const double rn2 = hred(c, b, 0);
        if (!std::isfinite(rn2)) {
            if (c->nb == 1) return fail(c, DMG_ENAN, "residual norm is not finite after step %d", step);
            return fail(c, DMG_ENAN, "residual norm of sample %d is not finite after step %d", b, step);
        }
        const double rel = std::sqrt(rn2) / P.nf[b];
        c->brel[b] = rel;
        c->bcyc[b] = step * cycles;
        worst = std::max(worst, rel);
        if (!fixed && (rel <= c->p.rtol || rn2 == 0.0)) {
            c->hact[b] = 0;
            P.active--;
            changed = true;
        }
    }
    if (info && step - 1 < DMG_HIST_LEN) info->hist[step - 1] = worst;
    if (info) info->outer = step;
    done = fixed || P.active == 0;
    if (changed && !done) TRY(push_act(c, s));
    return DMG_OK;
}

// Selects the launch variant for the next step: 0 while every sample iterates
// (kernels get no mask), 1 once some sample is done (kernels read act). Sets
// the mask argument the launches issued from now on carry.
int use_mask(dmg_ctx *c, const Progress &P) {
    const int m = P.active < c->nb ? 1 : 0;
    c->mask = m ? c->act : nullptr;
    return m;
}

// summary over the batch: most cycles, largest final relative residual
dmg_status progress_end(dmg_ctx *c, dmg_info *info) {
    int cyc = 0;
    double worst = 0.0;
    for (int b = 0; b < c->nb; b++) {
        cyc = std::max(cyc, c->bcyc[b]);
        worst = std::max(worst, c->brel[b]);
    }
    if (info) { info->cycles = cyc; info->rel_residual = worst; }
    for (int b = 0; b < c->nb; b++)
        if (c->brel[b] > c->p.rtol) {
            if (c->nb == 1)
                return fail(c, DMG_ENOCONV, "relative residual %.3e > rtol %.3e after %d cycles", c->brel[b],
                            c->p.rtol, c->bcyc[b]);
            return fail(c, DMG_ENOCONV, "sample %d: relative residual %.3e > rtol %.3e after %d cycles", b,
                        c->brel[b], c->p.rtol, c->bcyc[b]);
        }
    return DMG_OK;
}

// Plain FP64 iteration on level 0: u_0 = 0, then V-cycles on A u_0 = f_0.
// fixed > 0: exactly `fixed` cycles; else until rtol or max_cycles. One graph
// replay per cycle (the cycle, and in tolerance mode the residual norm and its
// read-back).
dmg_status iterate64(dmg_ctx *c, bool transposed, int fixed, dmg_info *info, cudaStream_t s) {
    Level &l = c->L[0];
    const int t = transposed ? 1 : 0;
    CUDA_TRY(c, cudaMemsetAsync(l.u, 0, l.n * sizeof(double), s));
    TRY(norm2_async(c, l.f, 0, s));
    TRY(finish_reduce(c, s));
    Progress P;
    TRY(progress_start(c, P, info, s));
    if (P.active == 0) return DMG_OK;
    bool done = false;
    if (fixed > 0) {
        const int m = use_mask(c, P);
        Graph &G = c->g_fix[t][m];
        TRY(capture(c, G, [&](cudaStream_t cs) { return vcycle<double>(c, 0, transposed, cs); }));
        for (int cyc = 1; cyc <= fixed; cyc++) {
            TRY(replay(c, G, s));
            if (c->prof_kernel >= 0 && !G.prof.empty()) {
                // each replay records the graph's event nodes anew: read them before the next
                CUDA_TRY(c, cudaStreamSynchronize(s));
                prof_harvest(c, G.prof, false);
            }
        }
        TRY(resid_norm_async(c, l.u, l.f, nullptr, 0, c->mask, s));
        TRY(finish_reduce(c, s));
        TRY(progress_step(c, P, 1, fixed, true, nullptr, done, s));
        if (info) { info->cycles = fixed; info->outer = fixed; }
        double worst = 0.0;
        for (double r : c->brel) worst = std::max(worst, r);
        if (info) info->rel_residual = worst;
        return DMG_OK;
    }
    for (int cyc = 1; cyc <= c->p.max_cycles && !done; cyc++) {
        Graph &G = c->g_cyc[t][use_mask(c, P)];
        TRY(capture(c, G, [&](cudaStream_t cs) -> dmg_status {
            TRY(vcycle<double>(c, 0, transposed, cs));
            TRY(resid_norm_async(c, l.u, l.f, nullptr, 0, c->mask, cs));
            return enqueue_readback(c, cs);
        }));
        TRY(replay(c, G, s));
        TRY(sync_read(c, s));
        prof_harvest(c, G.prof, false);
        TRY(progress_step(c, P, cyc, 1, false, info, done, s));
    }
    return progress_end(c, info);
}

// Mixed precision defect correction on level 0 (FP64 u_0, f_0): each step runs
// inner_cycles FP32 V-cycles on A e = r * 2^-e_cur from e = 0, then updates
// u_0 += e * 2^e_cur and forms the next FP64 residual and its norm. Residual,
// norms and update stay in FP64; the scale exponents live on the device, so a
// whole step is one graph replay.
dmg_status iterate_mixed(dmg_ctx *c, bool transposed, dmg_info *info, cudaStream_t s) {
    Level &l = c->L[0];
    const int t = transposed ? 1 : 0;
    CUDA_TRY(c, cudaMemsetAsync(l.u, 0, l.n * sizeof(double), s));
    TRY(norm2_async(c, l.f, 0, s));
    dmgk::k_mix_init<<<(c->nb + 127) / 128, 128, 0, s>>>(c->red, 0, c->ms, c->nb);
    TRY(check_launch(c, "mix_init"));
    dmgk::k_to_f32<<<grid_int_pair(l.g), blk(), 0, s>>>(l.g, l.f, c->ms, l.f32);
    TRY(check_launch(c, "to_f32"));
    TRY(finish_reduce(c, s));
    Progress P;
    TRY(progress_start(c, P, info, s));
    if (P.active == 0) return DMG_OK;
    bool done = false;
    for (int step = 1; step <= c->p.max_cycles && !done; step++) {
        Graph &G = c->g_mix[t][use_mask(c, P)];
        TRY(capture(c, G, [&](cudaStream_t cs) -> dmg_status {
            CUDA_TRY(c, cudaMemsetAsync(l.u32, 0, l.n * sizeof(float), cs));
            for (int ic = 0; ic < c->p.inner_cycles; ic++) TRY(vcycle<float>(c, 0, transposed, cs));
            dmgk::k_update<<<grid_int_pair(l.g), blk(), 0, cs>>>(l.g, l.u, l.u32, c->ms, c->mask);
            TRY(check_launch(c, "update"));
            TRY(resid_norm_async(c, l.u, l.f, l.f32, 0, c->mask, cs));
            dmgk::k_mix_next<<<(c->nb + 127) / 128, 128, 0, cs>>>(c->red, 0, c->ms, c->nb, c->mask);
            TRY(check_launch(c, "mix_next"));
            return enqueue_readback(c, cs);
        }));
        TRY(replay(c, G, s));
        TRY(sync_read(c, s));
        prof_harvest(c, G.prof, false);
        TRY(progress_step(c, P, step, c->p.inner_cycles, false, info, done, s));
    }
    return progress_end(c, info);
}

dmg_status iterate(dmg_ctx *c, bool transposed, int fixed, dmg_info *info, cudaStream_t s) {
    if (fixed > 0 || c->p.precision == DMG_FP64) return iterate64(c, transposed, fixed, info, s);
    return iterate_mixed(c, transposed, info, s);
}

int count_levels(int nx, int ny, int nz) {
    if (nz == 1) {   // 2D: halve x and y while both have an odd count > 3
        if (nx < 3 || ny < 3) return 0;
        int n = 1;
        while (nx > 3 && ny > 3 && (nx & 1) && (ny & 1)) {
            nx = (nx - 1) / 2 + 1;
            ny = (ny - 1) / 2 + 1;
            if (++n > kMaxLevels) return 0;
        }
        return n;
    }
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

// Half-row pitch: the parity's vertex count rounded up to 32 elements (rows
// aligned for the warps' 256-byte accesses), unless that pads by more than a
// quarter (short rows: 65 -> 96 at 129^3), then to 8 (half-rows still start on
// a 32-byte sector; pairs stay 8- and 16-byte aligned). Measured: at 257^3 the
// 32-element pitch (160 against 136) gives the faster half-sweep, at 129^3 the
// 8-element one (72 against 96).
inline int half_row_pitch(int nx) {
    const int nh = (nx + 1) / 2, p32 = (nh + 31) / 32 * 32;
    return 4 * (p32 - nh) <= nh ? p32 : (nh + 7) / 8 * 8;
}

Geom make_geom(int nx, int ny, int nz, int nb) {
    Geom g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.hx = half_row_pitch(nx);
    g.sy = 2 * g.hx;
    g.sz = (long long)g.sy * ny;
    g.sb = g.sz * nz;
    g.nb = nb;
    for (int w = 0; w < 3; w++) {
        // a 2D grid (nz == 1) has no interior or cell planes: those entries are unused
        const long long d = (long long)nz - 2 + w;
        g.mz[w] = d <= 1 ? 0u : (unsigned)(((1ULL << 32) + (unsigned long long)d - 1) / (unsigned long long)d);
    }
    return g;
}

dmg_status validate(dmg_ctx *c, const dmg_params *p) {
    if (!p) return fail(c, DMG_EINVAL, "params is NULL");
    if (p->nx < 3 || p->ny < 3 || (p->nz < 3 && p->nz != 1))
        return fail(c, DMG_EINVAL, "grid %dx%dx%d: every axis needs >= 3 vertices (nz = 1: a 2D grid)", p->nx,
                    p->ny, p->nz);
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
    if (p->batch < 1) return fail(c, DMG_EINVAL, "batch must be >= 1");
    if (p->autotune != 0 && p->autotune != 1) return fail(c, DMG_EINVAL, "autotune must be 0 or 1");
    if (p->split_prolong != 0 && p->split_prolong != 1) return fail(c, DMG_EINVAL, "split_prolong must be 0 or 1");
    if (p->twin_adjoint != 0 && p->twin_adjoint != 1) return fail(c, DMG_EINVAL, "twin_adjoint must be 0 or 1");
    {
        const Geom g0 = make_geom(p->nx, p->ny, p->nz, 1);
        if (g0.sb > (long long)INT32_MAX)
            return fail(c, DMG_EINVAL, "grid %dx%dx%d: a padded sample of %lld elements exceeds 2^31 - 1", p->nx,
                        p->ny, p->nz, g0.sb);
    }
    if ((long long)p->batch * p->nz > 65535)
        return fail(c, DMG_EINVAL, "batch * nz = %lld exceeds 65535", (long long)p->batch * p->nz);
    int nl = count_levels(p->nx, p->ny, p->nz);
    if (nl == 0) return fail(c, DMG_EINVAL, "grid %dx%dx%d cannot be coarsened", p->nx, p->ny, p->nz);
    int cx = p->nx, cy = p->ny, cz = p->nz;
    for (int l = 1; l < nl; l++) { cx = (cx - 1) / 2 + 1; cy = (cy - 1) / 2 + 1; cz = (cz - 1) / 2 + 1; }
    long long nc = (long long)(cx - 2) * (cy - 2) * (p->nz == 1 ? 1 : cz - 2);
    if (nc > kMaxCoarse)
        return fail(c, DMG_EINVAL,
                    "grid %dx%dx%d coarsens to %dx%dx%d with %lld unknowns (> %d): use c*2^n+1 vertices with small c",
                    p->nx, p->ny, p->nz, cx, cy, cz, nc, kMaxCoarse);
    return DMG_OK;
}

// --- tile autotuner ----------------------------------------------------------------
// Chooses, per level and precision, the thread-block shape of the colour kernels
// (the half-sweep, whose shape the colour defect shares) by timing half-sweeps
// on the level's own arrays during setup. Results are kept for the process
// (keyed by device, precision, grid, batch and face mean) and, when the
// environment variable DMG_TUNE_CACHE names a file, read from and appended to
// it. A candidate replaces the level's default (32 x 8 for FP64; for the FP32
// pair kernels 32 x 4, 16 x 8 or 8 x 16 by the level's width) only when it is at
// least 3% faster.

// candidates per precision (timed after the level's default shape)
const dim3 kTiles[2][9] = {{dim3(32, 8), dim3(32, 4), dim3(32, 2), dim3(64, 4), dim3(64, 2), dim3(128, 2),
                            dim3(128, 1), dim3(16, 16), dim3(16, 8)},
                           {dim3(32, 4), dim3(32, 8), dim3(32, 2), dim3(64, 4), dim3(64, 2), dim3(16, 16),
                            dim3(16, 8), dim3(8, 16), dim3(8, 32)}};

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;
bool g_tune_loaded = false;

std::string tune_key(int prec, const Geom &g, int harm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        prop.name[0] = 0;
    }
    std::string name(prop.name);
    for (char &ch : name)
        if (ch == ' ') ch = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "%s:%s:%dx%dx%d:b%d:h%d", name.c_str(), prec ? "f32" : "f64", g.nx, g.ny, g.nz, g.nb,
             harm);
    return buf;
}

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("DMG_TUNE_CACHE");
    if (!path) return;
    FILE *fh = fopen(path, "r");
    if (!fh) return;
    char key[256];
    int bx, by;
    while (fscanf(fh, "%255s %d %d", key, &bx, &by) == 3)
        if (bx > 0 && by > 0 && bx * by <= 256) g_tune[key] = {bx, by};
    fclose(fh);
}

void tune_store_locked(const std::string &key, dim3 b) {
    g_tune[key] = {(int)b.x, (int)b.y};
    const char *path = getenv("DMG_TUNE_CACHE");
    if (!path) return;
    FILE *fh = fopen(path, "a");
    if (!fh) return;
    fprintf(fh, "%s %u %u\n", key.c_str(), b.x, b.y);
    fclose(fh);
}

// one half-sweep of level l with block shape b (precision 1: FP32 vertex kernel)
dmg_status tune_launch(dmg_ctx *c, int l, int prec, dim3 b, int color, cudaStream_t s) {
    Level &L = c->L[l];
    if (prec == 1) {
        return with_coef32(c, L, [&](auto cf) {
            constexpr bool H = decltype(cf)::harmonic;
            if (c->nb == 1)
                dmgk::k_smooth_half32<H, false><<<grid_pair(L.g, b), b, 0, s>>>(L.g, L.u32, L.f32, cf, color, nullptr);
            else
                dmgk::k_smooth_half32<H, true><<<grid_pair(L.g, b), b, 0, s>>>(L.g, L.u32, L.f32, cf, color, nullptr);
            return check_launch(c, "tune");
        });
    }
    dmgk::k_smooth_half<double><<<grid_half(L.g, b), b, 0, s>>>(L.g, L.u, L.f, coef64(L), color, nullptr);
    return check_launch(c, "tune");
}

dmg_status tune_level(dmg_ctx *c, int l, int prec, cudaStream_t s) {
    const std::string key = tune_key(prec, c->L[l].g, c->p.face_mean);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            c->tb[prec][l] = dim3(it->second.first, it->second.second);
            return DMG_OK;
        }
    }
    // the arrays hold zeros at setup: half-sweeps leave them zero
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    // the level's default shape first; a candidate must beat it by 3%
    const dim3 def = c->tb[prec][l];
    dim3 best = def;
    float best_ms = 0.f;
    dmg_status st = DMG_OK;
    const size_t ncand = sizeof(kTiles[0]) / sizeof(kTiles[0][0]);
    for (size_t q = 0; q <= ncand && st == DMG_OK; q++) {
        const dim3 b = q == 0 ? def : kTiles[prec][q - 1];
        if (q > 0 && b.x == def.x && b.y == def.y) continue;
        for (int w = 0; w < 2 && st == DMG_OK; w++) st = tune_launch(c, l, prec, b, w, s);
        if (st != DMG_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 8 && st == DMG_OK; r++) st = tune_launch(c, l, prec, b, r & 1, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = fail(c, DMG_ECUDA, "autotuner timing failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (q == 0) best_ms = ms;
        else if (ms < 0.97f * best_ms) { best = b; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != DMG_OK) return st;
    c->tb[prec][l] = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_store_locked(key, best);
    return DMG_OK;
}

dmg_status autotune(dmg_ctx *c, cudaStream_t s) {
    if (c->dim == 2) return DMG_OK;   // the 2D kernels use the default shape
    for (int l = 0; l < c->tail_first[0] && l < c->nlev - 1; l++) TRY(tune_level(c, l, 0, s));
    if (c->p.precision == DMG_MIXED)
        for (int l = 0; l < c->tail_first[1] && l < c->nlev - 1; l++) TRY(tune_level(c, l, 1, s));
    return DMG_OK;
}

// Samples [first, first + count) of level l (pointers at the first one's part)
Level level_range(const dmg_ctx *c, int l, int first, int count) {
    Level v = c->L[l];
    const long long o = (long long)first * v.g.sb;
    v.g.nb = count;
    v.n = (size_t)v.g.sb * count;
    for (double **q : {&v.u, &v.f, &v.r, &v.cx, &v.cy, &v.cz, &v.diag, &v.invd, &v.D, &v.mu})
        if (*q) *q += o;
    for (float **q : {&v.u32, &v.f32, &v.r32, &v.Dh32, &v.mu32})
        if (*q) *q += o;
    return v;
}

// Level l of one slot (a single sample, pointers at its part; slot < 0: the
// level itself with every sample).
Level level_view(const dmg_ctx *c, int l, int slot) {
    if (slot < 0) return c->L[l];
    return level_range(c, l, slot, 1);
}

// a slot's finest level and its outputs there (U0: forward solution, T1, T2:
// tangent coefficients or gradients)
struct SlotTop {
    int lev;
    Level v;
    double *U0, *T1, *T2;
};
SlotTop slot_top(const dmg_ctx *c, int slot) {
    SlotTop t;
    t.lev = c->top_of[slot];
    t.v = level_view(c, t.lev, slot);
    t.v.h = c->p.h;   // every slot's finest grid has the spacing h
    const long long o = (long long)(slot - c->top_first[t.lev]) * t.v.g.sb;
    t.U0 = c->U0l[t.lev] + o;
    t.T1 = c->T1l[t.lev] + o;
    t.T2 = c->T2l[t.lev] + o;
    return t;
}

// The coefficient hierarchy of every sample (slot < 0) or of one slot
// (Sec. 2.2: D and mu coarsened level by level, the operator rediscretised on
// every level, the coarsest one inverted). Asynchronous; the Gauss-Jordan
// status of each built sample lands in hstatus once the stream reaches it.
dmg_status build_coefficients(dmg_ctx *c, int slot, const double *D, const double *mu, cudaStream_t s) {
    const dmg_params *p = &c->p;
    const bool mixed = p->precision == DMG_MIXED;
    Level V[kMaxLevels];
    // a slot's hierarchy starts at its finest level (0 unless the context is a pyramid)
    const int l0 = slot < 0 ? 0 : c->top_of[slot];
    for (int l = l0; l < c->nlev; l++) V[l] = level_view(c, l, slot);
    TRY(stage_in(c, D, V[l0].D, false, s, slot));
    TRY(stage_in(c, mu, V[l0].mu, false, s, slot));
    for (int l = l0 + 1; l < c->nlev; l++) {
        Level &F = V[l - 1], &C = V[l];
        if (c->dim == 2) {
            dmgk::k_coarsen2<<<grid_all2(C.g), blk(), 0, s>>>(F.g, F.D, C.g, C.D, p->coarsen);
            TRY(check_launch(c, "coarsen"));
            dmgk::k_coarsen2<<<grid_all2(C.g), blk(), 0, s>>>(F.g, F.mu, C.g, C.mu, p->coarsen);
            TRY(check_launch(c, "coarsen"));
            continue;
        }
        dmgk::k_coarsen<<<grid_all(C.g), blk(), 0, s>>>(F.g, F.D, C.g, C.D, p->coarsen);
        TRY(check_launch(c, "coarsen"));
        dmgk::k_coarsen<<<grid_all(C.g), blk(), 0, s>>>(F.g, F.mu, C.g, C.mu, p->coarsen);
        TRY(check_launch(c, "coarsen"));
    }
    const int harm = p->face_mean == DMG_FACE_HARMONIC;
    for (int l = l0; l < c->nlev; l++) {
        Level &L = V[l];
        // spacing of level l for these samples: h on the slot's finest level,
        // doubling per level below it (a pyramid's levels serve grids of one h)
        const double hl = std::ldexp(c->p.h, l - l0);
        const double ih2 = 1.0 / (hl * hl);
        if (c->dim == 2)
            dmgk::k_build_faces2<<<grid_all2(L.g), blk(), 0, s>>>(L.g, L.D, L.mu, ih2, harm, L.cx, L.cy, L.diag,
                                                                  L.invd);
        else
            dmgk::k_build_faces<<<grid_all(L.g), blk(), 0, s>>>(L.g, L.D, L.mu, ih2, harm, L.cx, L.cy, L.cz,
                                                                L.diag, L.invd);
        TRY(check_launch(c, "build_faces"));
        if (mixed) {
            const double scale = harm ? ih2 : 0.5 * ih2;
            dmgk::k_build_vertex32<<<grid_all(L.g), blk(), 0, s>>>(L.g, L.D, L.mu, scale, L.Dh32, L.mu32);
            TRY(check_launch(c, "build_vertex32"));
        }
    }
    const Level &LC = V[c->nlev - 1];
    const size_t nc2 = (size_t)c->nc * c->nc;
    const int first = slot < 0 ? 0 : slot, count = slot < 0 ? c->nb : 1;
    CUDA_TRY(c, cudaMemsetAsync(c->gj_status + first, 0xff, count * sizeof(int), s));
    if (c->dim == 2)
        dmgk::k_coarse_assemble2<<<dim3(64, count), 256, 0, s>>>(LC.g, coef64(LC), c->nc, c->M + 2 * nc2 * first);
    else
        dmgk::k_coarse_assemble<<<dim3(64, count), 256, 0, s>>>(LC.g, coef64(LC), c->nc, c->M + 2 * nc2 * first);
    TRY(check_launch(c, "coarse_assemble"));
    dmgk::k_gauss_jordan<<<count, 1024, 0, s>>>(c->M + 2 * nc2 * first, c->nc, c->Ainv + nc2 * first,
                                                c->Ainv32 + nc2 * first, c->gj_status + first);
    TRY(check_launch(c, "gauss_jordan"));
    CUDA_TRY(c, cudaMemcpyAsync(c->hstatus + first, c->gj_status + first, count * sizeof(int),
                                cudaMemcpyDeviceToHost, s));
    TRY(build_tail_image<double>(c, first, count, s));
    if (mixed) TRY(build_tail_image<float>(c, first, count, s));
    return DMG_OK;
}

// per_level (pyramid pools only): per_level[k] slots have level k as their
// finest level, k < nper; D and mu are then not read (slots are loaded one by one)
dmg_status setup_impl(dmg_ctx *c, const dmg_params *p, const double *D, const double *mu, cudaStream_t s,
                      const int *per_level = nullptr, int nper = 0) {
    dmg_params pp;
    if (per_level) {
        if (!p) return fail(c, DMG_EINVAL, "params is NULL");
        const int nl = count_levels(p->nx, p->ny, p->nz);
        if (p->nz == 1) return fail(c, DMG_EINVAL, "pyramid pools are 3D only");
        if (nper < 1 || nper > nl) return fail(c, DMG_EINVAL, "nlevels must be in [1, %d]", nl);
        long long total = 0;
        for (int k = 0; k < nper; k++) {
            if (per_level[k] < 0) return fail(c, DMG_EINVAL, "slots_per_level[%d] < 0", k);
            total += per_level[k];
        }
        if (total < 1 || total > 65535) return fail(c, DMG_EINVAL, "a pyramid needs 1 to 65535 slots");
        pp = *p;
        pp.batch = (int)total;
        p = &pp;
    }
    TRY(validate(c, p));
    if (!per_level && (!D || !mu)) return fail(c, DMG_EINVAL, "D and mu must not be NULL");
    c->p = *p;
    c->nb = p->batch;
    const int nb = c->nb;
    for (dim3 &b : c->tb[0]) b = dim3(32, 8, 1);
    c->nlev = count_levels(p->nx, p->ny, p->nz);
    c->dim = p->nz == 1 ? 2 : 3;
    c->pyramid = per_level != nullptr;
    // samples per level and the slots whose finest level each level is
    int nb_at[kMaxLevels];
    {
        int acc = 0;
        for (int l = 0; l < c->nlev; l++) {
            c->top_first[l] = acc;
            c->top_count[l] = per_level ? (l < nper ? per_level[l] : 0) : (l == 0 ? nb : 0);
            acc += c->top_count[l];
            nb_at[l] = acc;
        }
        c->top_of.assign(nb, 0);
        for (int l = 0; l < c->nlev; l++)
            for (int b = c->top_first[l]; b < c->top_first[l] + c->top_count[l]; b++) c->top_of[b] = l;
    }
    bool mixed = p->precision == DMG_MIXED;
    for (int l = 0; l < c->nlev; l++) {
        Level &L = c->L[l];
        if (l == 0) {
            L.g = make_geom(p->nx, p->ny, p->nz, nb_at[l]);
            L.h = p->h;
        } else {
            const Level &F = c->L[l - 1];
            L.g = make_geom((F.g.nx - 1) / 2 + 1, (F.g.ny - 1) / 2 + 1, (F.g.nz - 1) / 2 + 1, nb_at[l]);
            L.h = 2.0 * F.h;
        }
        if ((long long)nb_at[l] * L.g.nz > 65535)
            return fail(c, DMG_EINVAL, "level %d: samples * nz = %lld exceeds 65535", l,
                        (long long)nb_at[l] * L.g.nz);
        L.n = (size_t)L.g.sb * nb_at[l];
        if (L.n == 0) continue;   // a pyramid level above every slot
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
    // FP32 pair kernels: 128-thread blocks whose x extent covers a row's pairs
    // ((nx - 2) / 4 + 1 of them) with few idle lanes: 32 x 4 on wide levels,
    // 16 x 8 and 8 x 16 on narrow ones
    for (int l = 0; l < c->nlev; l++) {
        const int pairs = (c->L[l].g.nx - 2) / 4 + 1;
        const unsigned bx = pairs > 16 ? 32u : (pairs > 8 ? 16u : 8u);
        c->tb[1][l] = dim3(bx, 128 / bx, 1);
    }
    Level &L0 = c->L[0];
    // contiguous staging: every slot's field at its finest level, back to back
    {
        c->stage_off.assign(nb, 0);
        long long acc = 0;
        for (int b = 0; b < nb; b++) {
            c->stage_off[b] = acc;
            const Geom &g = c->L[c->top_of[b]].g;
            acc += (long long)g.nx * g.ny * g.nz;
        }
        TRY(dalloc(c, &c->stage, (size_t)acc));
        TRY(dalloc(c, &c->stage2, (size_t)acc));
    }
    if (!c->pyramid) {
        for (double **q : {&c->U0, &c->T1, &c->T2, &c->T3}) {
            TRY(dalloc(c, q, L0.n));
            CUDA_TRY(c, cudaMemsetAsync(*q, 0, L0.n * sizeof(double), s));
        }
        c->U0l[0] = c->U0;
        c->T1l[0] = c->T1;
        c->T2l[0] = c->T2;
    } else {
        for (int l = 0; l < c->nlev; l++) {
            const size_t n = (size_t)c->L[l].g.sb * c->top_count[l];
            if (n == 0) continue;
            for (double **q : {&c->U0l[l], &c->T1l[l], &c->T2l[l]}) {
                TRY(dalloc(c, q, n));
                CUDA_TRY(c, cudaMemsetAsync(*q, 0, n * sizeof(double), s));
            }
        }
        c->U0 = c->U0l[0];
    }
    TRY(dalloc(c, &c->partial, (size_t)kNormBlocks * nb));
    TRY(dalloc(c, &c->red, (size_t)kSlots * nb));
    TRY(dalloc(c, &c->ms, nb));
    TRY(dalloc(c, &c->act, nb));
    CUDA_TRY(c, cudaMemsetAsync(c->ms, 0, nb * sizeof(dmgk::MixScalars), s));
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_aux, cudaEventDisableTiming));
    CUDA_TRY(c, cudaMemsetAsync(c->red, 0, (size_t)kSlots * nb * sizeof(double), s));
    {
        // mapped pinned memory: kernels write the read-back and read the mask through the mapping
        cudaError_t e = cudaHostAlloc(&c->hred, (size_t)kSlots * nb * sizeof(double), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostAlloc(&c->hact, nb * sizeof(int), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&c->hred_d, c->hred, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&c->hact_d, c->hact, 0);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, DMG_ENOMEM, "cudaHostAlloc failed"); }
        memset(c->hred, 0, (size_t)kSlots * nb * sizeof(double));
        for (int b = 0; b < nb; b++) c->hact[b] = 1;
    }
    TRY(push_act(c, s));
    TRY(dalloc(c, &c->act_a, nb));
    CUDA_TRY(c, cudaMemsetAsync(c->act_a, 0, nb * sizeof(int), s));
    {
        cudaError_t e = cudaHostAlloc(&c->hact_a, nb * sizeof(int), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&c->hact_a_d, c->hact_a, 0);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, DMG_ENOMEM, "cudaHostAlloc failed"); }
        memset(c->hact_a, 0, nb * sizeof(int));
    }
    c->slots.assign(nb, Slot());
    for (Slot &sl : c->slots) sl.loaded = !c->pyramid;   // setup builds every sample's hierarchy (pyramid: none)
    c->bcyc.assign(nb, 0);
    c->brel.assign(nb, 0.0);
    Level &LC0 = c->L[c->nlev - 1];
    // coarsest unknowns (the tail sizes its buffer by it)
    c->nc = (LC0.g.nx - 2) * (LC0.g.ny - 2) * (c->dim == 2 ? 1 : LC0.g.nz - 2);
    // single-CTA tail: the small levels, as many as fit the shared-memory budget
    for (int t = 0; t < 2; t++) {
        const size_t esz = t ? sizeof(float) : sizeof(double);
        const int nops = t ? 4 : 5;   // operator arrays per level in the tail's image
        // the image of one sample (a multiple of 16 bytes) and the tail's shared memory
        auto img = [&](int first) {
            size_t e = 0;
            for (int l = first; l < c->nlev; l++) {
                Geom gs = smem_geom(c->L[l].g);
                e += (size_t)gs.sz * gs.nz * nops;
            }
            const size_t q = 16 / esz;
            return (e + q - 1) / q * q;
        };
        auto bytes = [&](int first) {
            size_t e = (size_t)c->nc + 16 + img(first);
            for (int l = first; l < c->nlev; l++) {
                Geom gs = smem_geom(c->L[l].g);
                e += (size_t)gs.sz * gs.nz * 3;
            }
            return e * esz;
        };
        int first = c->nlev - 1;
        while (first > 0) {
            const Geom &g = c->L[first - 1].g;
            if ((long long)(g.nx - 2) * (g.ny - 2) * (g.nz - 2) > kTailMaxInterior[t]) break;
            if (bytes(first - 1) > kTailSmemBudget) break;
            first--;
        }
        if (bytes(first) > kTailSmemBudget) first = c->nlev;   // even the coarsest does not fit: no tail
        if (c->dim == 2) first = c->nlev;   // the shared-memory tail is 3D only
        c->tail_first[t] = first;
        c->tail_smem[t] = first < c->nlev ? bytes(first) : 0;
        c->tail_img[t] = first < c->nlev ? (int)img(first) : 0;
    }
    if (c->tail_first[0] < c->nlev) TRY(dalloc(c, &c->timg64, (size_t)c->tail_img[0] * nb));
    if (mixed && c->tail_first[1] < c->nlev) TRY(dalloc(c, &c->timg32, (size_t)c->tail_img[1] * nb));
    if (c->pyramid) {
        // every slot's finest level lies above the single-CTA tail (which stages
        // the levels below from the coarse defects) and the coarsest level
        const int t = mixed ? 1 : 0;
        for (int l = 0; l < c->nlev; l++)
            if (c->top_count[l] > 0 && (l >= c->tail_first[t] || l >= c->nlev - 1))
                return fail(c, DMG_EINVAL,
                            "slots whose finest level is level %d (%dx%dx%d) would start inside the small-level "
                            "tail: use larger grids", l, c->L[l].g.nx, c->L[l].g.ny, c->L[l].g.nz);
    }
    {
        // the attribute belongs to the device's context: set it once per device
        static std::mutex mu;
        static bool done[256] = {false};
        int dev = 0;
        CUDA_TRY(c, cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 256 && !done[dev]) {
            for (auto fn : {(const void *)dmgk::k_vcycle_tail<double, dmgk::FaceCoef<double>>,
                            (const void *)dmgk::k_vcycle_tail<float, dmgk::VertCoef<float, false>>,
                            (const void *)dmgk::k_vcycle_tail<float, dmgk::VertCoef<float, true>>})
                CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kTailSmemBudget));
            done[dev] = true;
        }
    }
    // exact coarsest solve: dense SPD inverse of every sample by in-block Gauss-Jordan
    const size_t nc2 = (size_t)c->nc * c->nc;
    TRY(dalloc(c, &c->M, 2 * nc2 * nb));
    TRY(dalloc(c, &c->Ainv, nc2 * nb));
    TRY(dalloc(c, &c->Ainv32, nc2 * nb));
    TRY(dalloc(c, &c->gj_status, nb));
    {
        cudaError_t e = cudaMallocHost(&c->hstatus, nb * sizeof(int));
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, DMG_ENOMEM, "cudaMallocHost failed"); }
    }
    if (c->pyramid) {   // slots get their coefficients from dmg_slot_load
        CUDA_TRY(c, cudaStreamSynchronize(s));
        return DMG_OK;
    }
    TRY(build_coefficients(c, -1, D, mu, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (p->autotune) TRY(autotune(c, s));
    for (int b = 0; b < nb; b++)
        if (c->hstatus[b] != 0) {
            if (nb == 1)
                return fail(c, DMG_EINVAL, "coarsest-level matrix is not positive definite (need D > 0, mu >= 0)");
            return fail(c, DMG_EINVAL,
                        "coarsest-level matrix of sample %d is not positive definite (need D > 0, mu >= 0)", b);
        }
    return DMG_OK;
}

// --- a stream of fwd+VJP pairs with overlapped host transfers --------------------
dmg_status many_alloc(dmg_ctx *c) {
    if (c->many_ready) return DMG_OK;
    const size_t n = (size_t)c->p.nx * c->p.ny * c->p.nz * c->nb;
    for (int b = 0; b < 2; b++) {
        TRY(dalloc(c, &c->mi_stage[b], 2 * n));
        TRY(dalloc(c, &c->mo_stage[b], 4 * n));
    }
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->up, cudaStreamNonBlocking));
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->down, cudaStreamNonBlocking));
    for (int b = 0; b < 2; b++)
        for (cudaEvent_t *e : {&c->ev_in[b], &c->ev_used[b], &c->ev_ready_u[b], &c->ev_ready[b], &c->ev_out[b],
                               &c->ev_in_q[b], &c->ev_used_w[b], &c->ev_qb[b]})
            CUDA_TRY(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    c->many_ready = true;
    return DMG_OK;
}

// Pairs i = 0 .. npairs-1, each dmg_solve(q[i]) then the converged pull-back
// of w[i]. Host inputs are copied on the upload stream into one of two staging
// buffers one pair ahead; host outputs are laid out on the caller's stream into
// one of two staging buffers and copied out on the download stream while the
// next pair iterates. Device arrays are read and written in place.
dmg_status twin_ready(dmg_ctx *c, cudaStream_t s);

dmg_status solve_vjp_many_impl(dmg_ctx *c, int npairs, const double *const *q, const double *const *w,
                               double *const *u, double *const *qbar, double *const *Dbar, double *const *mubar,
                               dmg_info *info_fwd, dmg_info *info_adj, cudaStream_t s) {
    if (npairs < 1 || !q || !w) return fail(c, DMG_EINVAL, "npairs must be >= 1 and q, w not NULL");
    for (int i = 0; i < npairs; i++)
        if (!q[i] || !w[i]) return fail(c, DMG_EINVAL, "q[%d] and w[%d] must not be NULL", i, i);
    TRY(many_alloc(c));
    if (c->p.twin_adjoint) {
        // without device memory for the twin the pairs run in one lane
        const dmg_status tw = twin_ready(c, s);
        if (tw != DMG_OK && tw != DMG_ENOMEM) return tw;
        c->err[0] = 0;
    }
    dmg_ctx *t = c->twin;
    Level &l = c->L[0];
    const Geom g = geom0(c, -1);
    const size_t n = (size_t)g.nx * g.ny * g.nz * g.nb;
    const size_t bytes = n * sizeof(double);
    auto out_at = [](double *const *a, int i) { return a ? a[i] : nullptr; };
    // H2D copies of pair i's host inputs into mi_stage[i % 2], once pair i-2 has gathered from it
    auto upload = [&](int i) -> dmg_status {
        const int b = i % 2;
        CUDA_TRY(c, cudaStreamWaitEvent(c->up, c->ev_used[b], 0));
        CUDA_TRY(c, cudaStreamWaitEvent(c->up, c->ev_used_w[b], 0));
        if (!is_device_ptr(q[i]))
            CUDA_TRY(c, cudaMemcpyAsync(c->mi_stage[b], q[i], bytes, cudaMemcpyHostToDevice, c->up));
        CUDA_TRY(c, cudaEventRecord(c->ev_in_q[b], c->up));   // the forward solve can start
        if (!is_device_ptr(w[i]))
            CUDA_TRY(c, cudaMemcpyAsync(c->mi_stage[b] + n, w[i], bytes, cudaMemcpyHostToDevice, c->up));
        CUDA_TRY(c, cudaEventRecord(c->ev_in[b], c->up));
        return DMG_OK;
    };
    // lay src out into dst (device) or into the output staging slot, whose copy to
    // the host follows on the download stream
    auto put_on = [&](const double *src, double *dst, double *stage_slot, cudaStream_t st) -> dmg_status {
        if (is_device_ptr(dst)) {
            dmgk::k_scatter<<<quad_grid(g), blk(), 0, st>>>(g, src, dst);
            return check_launch(c, "scatter");
        }
        dmgk::k_scatter<<<quad_grid(g), blk(), 0, st>>>(g, src, stage_slot);
        return check_launch(c, "scatter");
    };
    auto put = [&](const double *src, double *dst, double *stage_slot) { return put_on(src, dst, stage_slot, s); };
    auto fetch = [&](const double *stage_slot, double *dst) -> dmg_status {
        if (dst && !is_device_ptr(dst))
            CUDA_TRY(c, cudaMemcpyAsync(dst, stage_slot, bytes, cudaMemcpyDeviceToHost, c->down));
        return DMG_OK;
    };
    const cudaStream_t caller = s;
    auto abort_all = [&](dmg_status st) {
        cudaStreamSynchronize(c->side);
        cudaStreamSynchronize(c->up);
        cudaStreamSynchronize(c->down);
        if (t) cudaStreamSynchronize(c->lead_s);
        return st;
    };
    dmg_status worst = DMG_OK;
    CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));   // the uploads start after the caller's earlier work
    CUDA_TRY(c, cudaStreamWaitEvent(c->up, c->ev_fork, 0));
    if (t) {
        // with two lanes the forward solves run on the high-priority stream
        CUDA_TRY(c, cudaStreamWaitEvent(c->lead_s, c->ev_fork, 0));
        s = c->lead_s;
    }
    TRY(upload(0));
    for (int i = 0; i < npairs; i++) {
        const int b = i % 2;
        double *mo = c->mo_stage[b];
        // inputs of pair i
        const double *qs = is_device_ptr(q[i]) ? q[i] : c->mi_stage[b];
        const double *ws = is_device_ptr(w[i]) ? w[i] : c->mi_stage[b] + n;
        if (t) {
            // two lanes: the forward solve starts once q is in, the adjoint one (in
            // the twin, on its own stream) once w is
            CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_in_q[b], 0));
            dmgk::k_gather<<<quad_grid(g), blk(), 0, s>>>(g, qs, l.f, 0);
            TRY(check_launch(c, "gather"));
            CUDA_TRY(c, cudaEventRecord(c->ev_used[b], s));
            CUDA_TRY(c, cudaStreamWaitEvent(c->twin_s, c->ev_in[b], 0));
            CUDA_TRY(c, cudaStreamWaitEvent(c->twin_s, c->ev_aux, 0));   // pair i-1's lam copied out
            dmgk::k_gather<<<quad_grid(g), blk(), 0, c->twin_s>>>(g, ws, t->L[0].f, 0);
            TRY(check_launch(c, "gather"));
            CUDA_TRY(c, cudaEventRecord(c->ev_used_w[b], c->twin_s));
        } else {
            CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_in[b], 0));
            dmgk::k_gather<<<quad_grid(g), blk(), 0, s>>>(g, qs, l.f, 0);
            TRY(check_launch(c, "gather"));
            dmgk::k_gather<<<quad_grid(g), blk(), 0, s>>>(g, ws, c->T3, 0);
            TRY(check_launch(c, "gather"));
            CUDA_TRY(c, cudaEventRecord(c->ev_used[b], s));
        }
        if (i + 1 < npairs) TRY(upload(i + 1));   // overlaps this pair's iterations
        if (t) {
            // the adjoint solve in the twin beside the forward one (see solve_vjp_twin)
            dmg_status st2 = DMG_OK;
            dmg_info *ia = info_adj ? info_adj + i : nullptr;
            double *const qb_i = out_at(qbar, i);
            double *const mo_i = mo;
            auto adjoint = [&]() {
                st2 = iterate(t, true, 0, ia, c->twin_s);
                if (st2 != DMG_OK && st2 != DMG_ENOCONV) return;
                // qbar = lam leaves as soon as the adjoint solve ends (the forward one is
                // longer), through its staging slot once pair i-2 has freed it
                if (!qb_i) return;
                cudaError_t e = cudaStreamWaitEvent(c->twin_s, c->ev_out[b], 0);
                const bool dev = is_device_ptr(qb_i);
                if (e == cudaSuccess) {
                    dmgk::k_scatter<<<quad_grid(g), blk(), 0, c->twin_s>>>(g, t->L[0].u, dev ? qb_i : mo_i + n);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess && !dev) {
                    e = cudaEventRecord(c->ev_qb[b], c->twin_s);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->down, c->ev_qb[b], 0);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(qb_i, mo_i + n, bytes, cudaMemcpyDeviceToHost, c->down);
                }
                if (e != cudaSuccess) st2 = fail(t, DMG_ECUDA, "read-out of qbar: %s", cudaGetErrorString(e));
            };
            std::thread lane;
            bool threaded = true;
            try {
                lane = std::thread(adjoint);
            } catch (...) {
                threaded = false;
            }
            dmg_status st = iterate(c, false, c->p.fixed_cycles, info_fwd ? info_fwd + i : nullptr, s);
            if (threaded) lane.join();
            else adjoint();
            if (st2 != DMG_OK && st2 != DMG_ENOCONV) {
                cudaStreamSynchronize(c->twin_s);
                return abort_all(fail(c, st2, "adjoint solve of pair %d: %s", i, t->err));
            }
            if (st != DMG_OK && st != DMG_ENOCONV) {
                cudaStreamSynchronize(c->twin_s);
                return abort_all(st);
            }
            if (st != DMG_OK || st2 != DMG_OK) worst = DMG_ENOCONV;
            CUDA_TRY(c, cudaEventRecord(c->ev_twin, c->twin_s));
            CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_twin, 0));
            // u and lam into U0 and T3 (once the side stream is done with pair i-1's),
            // so that the next pair's solves can start while this pair's gradients and
            // read-out run on the side stream
            CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_join, 0));
            TRY(dcopy(c, c->U0, l.u, l.n, s));
            TRY(dcopy(c, c->T3, t->L[0].u, l.n, s));
            CUDA_TRY(c, cudaEventRecord(c->ev_aux, s));
            cudaStream_t sd = c->side;
            CUDA_TRY(c, cudaStreamWaitEvent(sd, c->ev_aux, 0));
            double *Db = out_at(Dbar, i), *mb = out_at(mubar, i), *ud = out_at(u, i);
            // the staging slot of pair i-2 must have reached the host
            CUDA_TRY(c, cudaStreamWaitEvent(sd, c->ev_out[b], 0));
            // the tiled gradient kernels (arithmetic face mean) write the natural
            // layout: into a device array itself, or into a host array's staging slot
            const bool harm = c->p.face_mean == DMG_FACE_HARMONIC, direct = grad_tiled(harm);
            if (Db || mb) {
                const double ih2 = 1.0 / (l.h * l.h);
                double *Dt = Db ? (direct ? (is_device_ptr(Db) ? Db : mo + 2 * n) : c->T1) : nullptr;
                double *mt = mb ? (direct ? (is_device_ptr(mb) ? mb : mo + 3 * n) : c->T2) : nullptr;
                ProfScope ps(c, DMG_KERNEL_GRAD, 0, 0, sd);
                if (c->dim == 2)
                    launch_grad2(sd, l.g, c->U0, c->T3, l.D, ih2, harm, Dt, mt, direct, direct);
                else
                    launch_grad(sd, l.g, c->U0, c->T3, l.D, ih2, harm, Dt, mt, direct, direct);
                TRY(check_launch(c, "grad"));
            }
            if (ud) TRY(put_on(c->U0, ud, mo, sd));
            if (Db && !direct) TRY(put_on(c->T1, Db, mo + 2 * n, sd));
            if (mb && !direct) TRY(put_on(c->T2, mb, mo + 3 * n, sd));
            CUDA_TRY(c, cudaEventRecord(c->ev_join, sd));   // U0, T3, T1, T2 free again
            CUDA_TRY(c, cudaEventRecord(c->ev_ready[b], sd));
            CUDA_TRY(c, cudaStreamWaitEvent(c->down, c->ev_ready[b], 0));
            if (ud) TRY(fetch(mo, ud));   // overlap the next pair's iterations
            if (Db) TRY(fetch(mo + 2 * n, Db));
            if (mb) TRY(fetch(mo + 3 * n, mb));
            CUDA_TRY(c, cudaEventRecord(c->ev_out[b], c->down));
            continue;
        }
        dmg_status st = iterate(c, false, c->p.fixed_cycles, info_fwd ? info_fwd + i : nullptr, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return abort_all(st);
        if (st != DMG_OK) worst = st;
        TRY(dcopy(c, c->U0, l.u, l.n, s));
        TRY(dcopy(c, l.f, c->T3, l.n, s));
        // the staging slot of pair i-2 must have reached the host
        CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_out[b], 0));
        if (double *dst = out_at(u, i)) {
            TRY(put(c->U0, dst, mo));
            CUDA_TRY(c, cudaEventRecord(c->ev_ready_u[b], s));
            CUDA_TRY(c, cudaStreamWaitEvent(c->down, c->ev_ready_u[b], 0));
            TRY(fetch(mo, dst));   // overlaps the adjoint iteration
        }
        st = iterate(c, true, 0, info_adj ? info_adj + i : nullptr, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return abort_all(st);
        if (st != DMG_OK) worst = st;
        double *Db = out_at(Dbar, i), *mb = out_at(mubar, i), *qb = out_at(qbar, i);
        if (Db || mb) {
            const double ih2 = 1.0 / (l.h * l.h);
            ProfScope ps(c, DMG_KERNEL_GRAD, 0, 0, s);
            if (c->dim == 2)
                launch_grad2(s, l.g, c->U0, l.u, l.D, ih2,
                                                               c->p.face_mean == DMG_FACE_HARMONIC,
                                                               Db ? c->T1 : nullptr, mb ? c->T2 : nullptr);
            else
                launch_grad(s, l.g, c->U0, l.u, l.D, ih2,
                                                             c->p.face_mean == DMG_FACE_HARMONIC,
                                                             Db ? c->T1 : nullptr, mb ? c->T2 : nullptr);
            TRY(check_launch(c, "grad"));
        }
        if (qb) TRY(put(l.u, qb, mo + n));
        if (Db) TRY(put(c->T1, Db, mo + 2 * n));
        if (mb) TRY(put(c->T2, mb, mo + 3 * n));
        CUDA_TRY(c, cudaEventRecord(c->ev_ready[b], s));
        CUDA_TRY(c, cudaStreamWaitEvent(c->down, c->ev_ready[b], 0));
        if (qb) TRY(fetch(mo + n, qb));   // overlap the next pair's iterations
        if (Db) TRY(fetch(mo + 2 * n, Db));
        if (mb) TRY(fetch(mo + 3 * n, mb));
        CUDA_TRY(c, cudaEventRecord(c->ev_out[b], c->down));
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->side));
    CUDA_TRY(c, cudaStreamSynchronize(c->up));
    CUDA_TRY(c, cudaStreamSynchronize(c->down));
    if (t) {
        CUDA_TRY(c, cudaEventRecord(c->ev_lead, c->lead_s));
        CUDA_TRY(c, cudaStreamWaitEvent(caller, c->ev_lead, 0));
    }
    TRY(end_call(c, caller));
    return worst;
}

// --- slot-level (serving) interface ---------------------------------------------
// A batched context doubles as a pool of slots. Each slot holds one request's
// coefficient hierarchy and runs one phase at a time (forward solve, tangent
// solve, adjoint solve); every step launch advances all running slots by one
// refinement step (mixed) or V-cycle (FP64), the forward-type phases in one
// graph and the adjoint phases in another, each masked to its slots. A slot's
// arithmetic is that of its sample alone, so a served result is bit for bit
// the result of dmg_solve/dmg_jvp/dmg_vjp on a context of batch 1.

bool slot_busy(const Slot &sl) { return sl.run == kStarting || sl.run == kRunning; }

bool any_busy(const dmg_ctx *c) {
    for (const Slot &sl : c->slots)
        if (slot_busy(sl)) return true;
    return false;
}

// calls on the whole context (every sample at level 0): not while slots run
// phases, and not on a pyramid pool, whose slots live on different levels
dmg_status need_whole(dmg_ctx *c) {
    if (c->pyramid) return fail(c, DMG_EINVAL, "a pyramid pool serves its slots only (dmg_slot_* calls)");
    if (any_busy(c)) return fail(c, DMG_EINVAL, "slots are running phases");
    return DMG_OK;
}

dmg_status check_slot(dmg_ctx *c, int slot) {
    if (c->dim == 2) return fail(c, DMG_EINVAL, "the slot interface is 3D only");
    if (slot < 0 || slot >= c->nb) return fail(c, DMG_EINVAL, "slot %d out of range [0, %d)", slot, c->nb);
    if (c->p.fixed_cycles != 0) return fail(c, DMG_EINVAL, "the slot interface needs fixed_cycles == 0");
    return DMG_OK;
}

dmg_status slot_load_impl(dmg_ctx *c, int slot, const double *D, const double *mu, cudaStream_t s) {
    TRY(check_slot(c, slot));
    if (!D || !mu) return fail(c, DMG_EINVAL, "D and mu must not be NULL");
    Slot &sl = c->slots[slot];
    if (slot_busy(sl)) return fail(c, DMG_EINVAL, "slot %d is running a phase", slot);
    TRY(build_coefficients(c, slot, D, mu, s));
    sl = Slot();
    sl.load_pending = true;
    return DMG_OK;
}

// New coefficients for every sample of an existing context: the hierarchy is
// rebuilt in place (the same kernels as setup, no allocation), so the
// context's graphs and buffers stay valid. Waits for the stream to check that
// every coarsest matrix is positive definite.
dmg_status set_coefficients_impl(dmg_ctx *c, const double *D, const double *mu, cudaStream_t s) {
    if (!D || !mu) return fail(c, DMG_EINVAL, "D and mu must not be NULL");
    TRY(need_whole(c));
    if (c->twin) {
        const dmg_status st = set_coefficients_impl(c->twin, D, mu, s);
        if (st != DMG_OK) return fail(c, st, "%s", c->twin->err);
    }
    TRY(build_coefficients(c, -1, D, mu, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    for (Slot &sl : c->slots) {
        sl = Slot();
        sl.loaded = true;
    }
    for (int b = 0; b < c->nb; b++)
        if (c->hstatus[b] != 0) {
            if (c->nb == 1)
                return fail(c, DMG_EINVAL, "coarsest-level matrix is not positive definite (need D > 0, mu >= 0)");
            return fail(c, DMG_EINVAL,
                        "coarsest-level matrix of sample %d is not positive definite (need D > 0, mu >= 0)", b);
        }
    return DMG_OK;
}

dmg_status destroy_impl(dmg_ctx *c);

// The twin of a context: the same parameters and coefficient hierarchy (built
// again from level 0's D and mu), its own iteration state, graphs and streams,
// so that an adjoint solve can run in it while the context solves forward.
dmg_status twin_ready(dmg_ctx *c, cudaStream_t s) {
    if (c->twin) return DMG_OK;
    const Geom g = c->L[0].g;
    const size_t n = (size_t)g.nx * g.ny * g.nz * g.nb;
    double *Dd = nullptr, *md = nullptr;
    cudaError_t e = cudaMalloc(&Dd, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&md, n * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(Dd);
        return fail(c, DMG_ENOMEM, "twin context: cudaMalloc of %zu bytes failed", 2 * n * sizeof(double));
    }
    dmgk::k_scatter<<<quad_grid(g), blk(), 0, s>>>(g, c->L[0].D, Dd);
    dmgk::k_scatter<<<quad_grid(g), blk(), 0, s>>>(g, c->L[0].mu, md);
    dmg_status st = check_launch(c, "scatter");
    dmg_ctx *t = nullptr;
    if (st == DMG_OK) {
        t = new (std::nothrow) dmg_ctx();
        if (!t) st = fail(c, DMG_ENOMEM, "twin context: out of host memory");
    }
    if (st == DMG_OK) {
        dmg_params p = c->p;
        p.autotune = 0;   // the context's tiles are copied below
        p.twin_adjoint = 0;
        st = setup_impl(t, &p, Dd, md, s);
        if (st != DMG_OK) st = fail(c, st, "twin context: %s", t->err);
    }
    if (st == DMG_OK) {
        memcpy(t->tb, c->tb, sizeof(c->tb));
        // the forward solve is the longer lane: its kernels go first where both lanes
        // have blocks waiting, and the adjoint lane fills the rest of the GPU
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->twin_s, cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->lead_s, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_twin, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_lead, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            st = fail(c, DMG_ECUDA, "twin context: stream or event creation failed");
            // a later call starts again from none of them
            for (cudaStream_t *x : {&c->twin_s, &c->lead_s})
                if (*x) {
                    cudaStreamDestroy(*x);
                    *x = nullptr;
                }
            for (cudaEvent_t *x : {&c->ev_twin, &c->ev_lead})
                if (*x) {
                    cudaEventDestroy(*x);
                    *x = nullptr;
                }
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(Dd);
    cudaFree(md);
    if (st != DMG_OK) {
        if (t) destroy_impl(t);
        return st;
    }
    c->twin = t;
    return DMG_OK;
}

// Forward solve and VJP with the adjoint solve A^T lam = w in the twin, on its
// own stream and host thread, while the forward one runs here; the gradient
// kernel then reads u from this context and lam from the twin.
dmg_status solve_vjp_twin(dmg_ctx *c, const double *q, const double *w, double *u, double *qbar, double *Dbar,
                          double *mubar, dmg_info *info_fwd, dmg_info *info_adj, cudaStream_t s) {
    dmg_ctx *t = c->twin;
    Level &l = c->L[0];
    CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));   // both lanes start after the caller's earlier work
    CUDA_TRY(c, cudaStreamWaitEvent(c->twin_s, c->ev_fork, 0));
    CUDA_TRY(c, cudaStreamWaitEvent(c->lead_s, c->ev_fork, 0));
    dmg_status st2 = DMG_OK;
    auto adjoint = [&]() {
        st2 = stage_in(t, w, t->L[0].f, false, c->twin_s);
        if (st2 == DMG_OK) st2 = iterate(t, true, 0, info_adj, c->twin_s);
        if (st2 != DMG_OK && st2 != DMG_ENOCONV) return;
        // lam is ready for the gradient kernel; qbar = lam leaves while the forward
        // lane still iterates (the adjoint solve is the shorter one)
        if (cudaEventRecord(c->ev_twin, c->twin_s) != cudaSuccess) {
            cudaGetLastError();
            st2 = fail(t, DMG_ECUDA, "event record failed");
            return;
        }
        if (qbar) {
            const dmg_status so = stage_out(t, t->L[0].u, qbar, c->twin_s);
            if (so != DMG_OK) st2 = so;
        }
    };
    std::thread lane;
    bool threaded = true;
    try {
        lane = std::thread(adjoint);
    } catch (...) {
        threaded = false;   // no thread: the adjoint runs after the forward solve
    }
    dmg_status st = stage_in(c, q, l.f, false, c->lead_s);
    if (st == DMG_OK) st = iterate(c, false, c->p.fixed_cycles, info_fwd, c->lead_s);
    if (threaded) lane.join();
    else adjoint();
    if (cudaEventRecord(c->ev_lead, c->lead_s) == cudaSuccess) cudaStreamWaitEvent(s, c->ev_lead, 0);
    if (st2 != DMG_OK && st2 != DMG_ENOCONV) {
        cudaStreamSynchronize(c->twin_s);
        cudaStreamSynchronize(c->lead_s);
        cudaStreamSynchronize(s);
        return fail(c, st2, "adjoint solve: %s", t->err);
    }
    if (st != DMG_OK && st != DMG_ENOCONV) {
        cudaStreamSynchronize(c->twin_s);
        cudaStreamSynchronize(c->lead_s);
        return st;
    }
    if (st == DMG_OK && st2 == DMG_ENOCONV) fail(c, st2, "adjoint solve: %s", t->err);
    CUDA_TRY(c, cudaEventRecord(c->ev_aux, c->twin_s));   // the lane's read-out of qbar ends
    CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_twin, 0));   // lam ready
    const double *lam = t->L[0].u;
    // u is read out on the side stream while the gradient kernel runs
    CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));
    CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    if (u) TRY(stage_out(c, l.u, u, c->side, -1, c->stage2));
    CUDA_TRY(c, cudaEventRecord(c->ev_join, c->side));
    if (Dbar || mubar) TRY(grad_out(c, l.u, lam, Dbar, mubar, s));
    CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_join, 0));
    CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_aux, 0));
    TRY(end_call(c, s));
    return st != DMG_OK ? st : st2;
}

dmg_status slot_begin_impl(dmg_ctx *c, int slot, int phase, const double *a, const double *b, const double *d,
                           cudaStream_t s) {
    TRY(check_slot(c, slot));
    Slot &sl = c->slots[slot];
    if (slot_busy(sl)) return fail(c, DMG_EINVAL, "slot %d is running a phase", slot);
    if (!sl.loaded && !sl.load_pending) return fail(c, DMG_EINVAL, "slot %d has no coefficients", slot);
    if (phase != DMG_PHASE_FORWARD && phase != DMG_PHASE_TANGENT && phase != DMG_PHASE_ADJOINT)
        return fail(c, DMG_EINVAL, "bad phase %d", phase);
    if ((phase == DMG_PHASE_FORWARD || phase == DMG_PHASE_ADJOINT) && !a)
        return fail(c, DMG_EINVAL, "the right-hand side must not be NULL");
    if (phase == DMG_PHASE_TANGENT && (b || d) && !sl.have_fwd)
        return fail(c, DMG_EINVAL, "slot %d has no forward solution for a D or mu tangent", slot);
    const SlotTop top = slot_top(c, slot);   // the slot's finest level
    const Level &l = top.v;
    CUDA_TRY(c, cudaMemsetAsync(l.u, 0, l.n * sizeof(double), s));
    if (a) {
        TRY(stage_in(c, a, l.f, false, s, slot));
    } else {
        CUDA_TRY(c, cudaMemsetAsync(l.f, 0, l.n * sizeof(double), s));
    }
    if (phase == DMG_PHASE_TANGENT && (b || d)) {
        if (b) TRY(stage_in(c, b, top.T1, false, s, slot));
        if (d) TRY(stage_in(c, d, top.T2, false, s, slot));
        const double ih2 = 1.0 / (l.h * l.h);
        dmgk::k_dA<<<grid_int(l.g), blk(), 0, s>>>(l.g, top.U0, b ? top.T1 : nullptr, d ? top.T2 : nullptr,
                                                   l.D, ih2, c->p.face_mean == DMG_FACE_HARMONIC, l.f);
        TRY(check_launch(c, "dA"));
    }
    // ||f||^2 -> red[slot][0]; mixed: the slot's scale and FP32 right-hand side
    dmgk::k_norm2<<<dim3(kNormBlocks, 1), 256, 0, s>>>(l.g, l.f, c->partial + (size_t)kNormBlocks * slot);
    TRY(check_launch(c, "norm2"));
    dmgk::k_reduce_final<<<1, 256, 0, s>>>(c->partial + (size_t)kNormBlocks * slot, kNormBlocks,
                                           c->red + (size_t)kSlots * slot, 0, nullptr);
    TRY(check_launch(c, "reduce"));
    if (c->p.precision == DMG_MIXED) {
        dmgk::k_mix_init<<<1, 32, 0, s>>>(c->red + (size_t)kSlots * slot, 0, c->ms + slot, 1);
        TRY(check_launch(c, "mix_init"));
        dmgk::k_to_f32<<<grid_int_pair(l.g), blk(), 0, s>>>(l.g, l.f, c->ms + slot, l.f32);
        TRY(check_launch(c, "to_f32"));
    }
    const bool keep_fwd = sl.have_fwd && phase != DMG_PHASE_FORWARD;
    const bool loaded = sl.loaded, pending = sl.load_pending, failed = sl.load_failed;
    sl = Slot();
    sl.loaded = loaded;
    sl.load_pending = pending;
    sl.load_failed = failed;
    sl.have_fwd = keep_fwd;
    sl.phase = phase;
    sl.run = kStarting;
    return DMG_OK;
}

// ||f - A u||^2 (FP64) of the slots whose finest level is lev -> red[slot][0];
// with r32: their FP32 right-hand sides r * 2^-e_prev
dmg_status top_resid_norm(dmg_ctx *c, int lev, bool r32, cudaStream_t s) {
    const int first = c->top_first[lev], cnt = c->top_count[lev];
    const Level v = level_range(c, lev, first, cnt);
    const int *act = c->mask ? c->mask + first : nullptr;
    {
        ProfScope ps(c, DMG_KERNEL_RESIDUAL, lev, 0, s);
        dmgk::k_resid_norm<double><<<dim3(kNormBlocks, cnt), 256, 0, s>>>(
            v.g, v.u, v.f, coef64(v), (double *)nullptr, r32 ? v.f32 : nullptr, c->ms + first,
            c->partial + (size_t)kNormBlocks * first, act);
        TRY(check_launch(c, "resid_norm"));
    }
    dmgk::k_reduce_final<<<cnt, 256, 0, s>>>(c->partial + (size_t)kNormBlocks * first, kNormBlocks,
                                             c->red + (size_t)kSlots * first, 0, act);
    return check_launch(c, "reduce");
}

// the step graph of one direction: t = 0 forward and tangent phases, 1 adjoint.
// In a pyramid the V-cycle starts at the finest level that holds slots and
// every level takes the samples it holds; each slot's refinement (update,
// residual, norm) runs on its own finest level.
dmg_status capture_step(dmg_ctx *c, int t) {
    const bool transposed = t == 1;
    c->mask = t ? c->act_a : c->act;
    int lev0 = 0;
    while (c->top_count[lev0] == 0) lev0++;
    return capture(c, c->g_srv[t], [&](cudaStream_t cs) -> dmg_status {
        if (c->p.precision == DMG_MIXED) {
            for (int lev = 0; lev < c->nlev; lev++) {
                if (c->top_count[lev] == 0) continue;
                const int first = c->top_first[lev];
                const Level v = level_range(c, lev, first, c->top_count[lev]);
                dmgk::k_zero_interior<float><<<grid_int(v.g), blk(), 0, cs>>>(v.g, v.u32,
                                                                              c->mask ? c->mask + first : nullptr);
                TRY(check_launch(c, "zero"));
            }
            for (int ic = 0; ic < c->p.inner_cycles; ic++) TRY(vcycle<float>(c, lev0, transposed, cs));
            for (int lev = 0; lev < c->nlev; lev++) {
                if (c->top_count[lev] == 0) continue;
                const int first = c->top_first[lev];
                const Level v = level_range(c, lev, first, c->top_count[lev]);
                dmgk::k_update<<<grid_int_pair(v.g), blk(), 0, cs>>>(v.g, v.u, v.u32, c->ms + first,
                                                                c->mask ? c->mask + first : nullptr);
                TRY(check_launch(c, "update"));
                TRY(top_resid_norm(c, lev, true, cs));
            }
            dmgk::k_mix_next<<<(c->nb + 127) / 128, 128, 0, cs>>>(c->red, 0, c->ms, c->nb, c->mask);
            return check_launch(c, "mix_next");
        }
        TRY(vcycle<double>(c, lev0, transposed, cs));
        for (int lev = 0; lev < c->nlev; lev++)
            if (c->top_count[lev] > 0) TRY(top_resid_norm(c, lev, false, cs));
        return DMG_OK;
    });
}

dmg_status step_launch_impl(dmg_ctx *c, cudaStream_t s) {
    if (c->step_open) return fail(c, DMG_EINVAL, "dmg_step_finish must follow every dmg_step_launch");
    bool run[2] = {false, false};
    for (int b = 0; b < c->nb; b++) {
        Slot &sl = c->slots[b];
        sl.in_step = sl.run == kRunning;
        sl.start_seen = sl.run == kStarting;
        const int t = sl.phase == DMG_PHASE_ADJOINT ? 1 : 0;
        c->hact[b] = sl.in_step && t == 0;
        c->hact_a[b] = sl.in_step && t == 1;
        if (sl.in_step) run[t] = true;
    }
    TRY(dcopy(c, c->act, (const int *)c->hact_d, (size_t)c->nb, s));
    TRY(dcopy(c, c->act_a, (const int *)c->hact_a_d, (size_t)c->nb, s));
    for (int t = 0; t < 2; t++) {
        if (!run[t]) continue;
        TRY(capture_step(c, t));
        TRY(replay(c, c->g_srv[t], s));
    }
    TRY(enqueue_readback(c, s));
    c->step_open = true;
    return DMG_OK;
}

void end_phase(dmg_ctx *c, int b, int status, std::vector<int> &ended) {
    Slot &sl = c->slots[b];
    sl.status = status;
    sl.run = kDone;
    ended.push_back(b);
}

dmg_status step_finish_impl(dmg_ctx *c, cudaStream_t s, int *ended_out, int *nended) {
    if (!c->step_open) return fail(c, DMG_EINVAL, "dmg_step_finish without dmg_step_launch");
    c->step_open = false;
    CUDA_TRY(c, cudaStreamSynchronize(s));
    prof_harvest(c, c->prof_direct, true);
    for (Graph &G : c->g_srv) prof_harvest(c, G.prof, false);
    std::vector<int> ended;
    const int per_step = c->p.precision == DMG_MIXED ? c->p.inner_cycles : 1;
    for (int b = 0; b < c->nb; b++) {
        Slot &sl = c->slots[b];
        if (sl.load_pending) {   // every load enqueued so far has completed
            sl.load_pending = false;
            sl.load_failed = c->hstatus[b] != 0;
            sl.loaded = !sl.load_failed;
        }
        if (slot_busy(sl) && sl.load_failed) {
            end_phase(c, b, DMG_EINVAL, ended);
            continue;
        }
        if (sl.run == kStarting && sl.start_seen) {
            const double n2 = hred(c, b, 0);
            sl.start_seen = false;
            if (!std::isfinite(n2)) {
                end_phase(c, b, DMG_ENAN, ended);
            } else if (n2 == 0.0) {
                sl.rel = 0.0;
                end_phase(c, b, DMG_OK, ended);
            } else {
                sl.nf = std::sqrt(n2);
                sl.rel = 1.0;
                sl.run = kRunning;
            }
        } else if (sl.run == kRunning && sl.in_step) {
            const double rn2 = hred(c, b, 0);
            sl.steps++;
            if (!std::isfinite(rn2)) {
                end_phase(c, b, DMG_ENAN, ended);
                continue;
            }
            sl.rel = std::sqrt(rn2) / sl.nf;
            if (sl.rel <= c->p.rtol || rn2 == 0.0) end_phase(c, b, DMG_OK, ended);
            else if (sl.steps >= c->p.max_cycles) end_phase(c, b, DMG_ENOCONV, ended);
        }
        sl.in_step = false;
    }
    // a finished forward phase leaves its solution in U0 for the tangent or adjoint phase
    for (int b : ended) {
        Slot &sl = c->slots[b];
        if (sl.phase == DMG_PHASE_FORWARD && (sl.status == DMG_OK || sl.status == DMG_ENOCONV)) {
            const SlotTop top = slot_top(c, b);
            TRY(dcopy(c, top.U0, (const double *)top.v.u, top.v.n, s));
            sl.have_fwd = true;
        }
        c->bcyc[b] = sl.steps * per_step;
        c->brel[b] = sl.rel;
    }
    if (nended) *nended = (int)ended.size();
    if (ended_out)
        for (size_t q = 0; q < ended.size(); q++) ended_out[q] = ended[q];
    return DMG_OK;
}

dmg_status slot_read_impl(dmg_ctx *c, int slot, double *u, double *x, double *Dbar, double *mubar,
                          cudaStream_t s) {
    TRY(check_slot(c, slot));
    Slot &sl = c->slots[slot];
    if (slot_busy(sl)) return fail(c, DMG_EINVAL, "slot %d is running a phase", slot);
    if (sl.phase < 0) return fail(c, DMG_EINVAL, "slot %d has run no phase", slot);
    if ((u || Dbar || mubar) && !sl.have_fwd) return fail(c, DMG_EINVAL, "slot %d has no forward solution", slot);
    if ((Dbar || mubar) && sl.phase != DMG_PHASE_ADJOINT)
        return fail(c, DMG_EINVAL, "Dbar and mubar need a finished adjoint phase");
    const SlotTop top = slot_top(c, slot);
    const Level &l = top.v;
    if (u) TRY(stage_out(c, top.U0, u, s, slot));
    if (x) TRY(stage_out(c, l.u, x, s, slot));
    if (Dbar || mubar) {
        const double ih2 = 1.0 / (l.h * l.h);
        ProfScope ps(c, DMG_KERNEL_GRAD, top.lev, 0, s);
        launch_grad(s, l.g, top.U0, l.u, l.D, ih2,
                                                     c->p.face_mean == DMG_FACE_HARMONIC,
                                                     Dbar ? top.T1 : nullptr, mubar ? top.T2 : nullptr);
        TRY(check_launch(c, "grad"));
        if (Dbar) TRY(stage_out(c, top.T1, Dbar, s, slot));
        if (mubar) TRY(stage_out(c, top.T2, mubar, s, slot));
    }
    return DMG_OK;
}

// --- unrolled coefficient gradient -------------------------------------------------
// The exact derivative of <w, S_m(q; D, mu)> for m FP64 V-cycles from u = 0,
// through every iterate and through the coarsened coefficients of every level.
// The forward cycles run with the grid kernels only (full defect, no
// single-CTA tail), so that every state the reverse pass needs can be saved.
// Iterates are recomputed from level-0 checkpoints taken every `stride` cycles:
// cycle c is rebuilt from the checkpoint at or before it and run once more
// saving its states, then reversed.

int n_states(const dmg_ctx *c) { return 2 * (c->p.nu1 + c->p.nu2) + 1; }

dmg_status unrolled_alloc(dmg_ctx *c, int nck) {
    // a failed attempt leaves un_ready false: the next call allocates a complete
    // set again (the partial one stays with the context until dmg_destroy)
    if (!c->un_ready) {
        for (int l = 0; l < c->nlev; l++) {
            ULevel &W = c->un[l];
            const size_t n = c->L[l].n;
            for (double **q : {&W.ub, &W.fb, &W.bx, &W.by, &W.bz, &W.mub, &W.Db, &W.tmp}) {
                TRY(dalloc(c, q, n));
                CUDA_TRY(c, cudaMemset(*q, 0, n * sizeof(double)));
            }
            const int ns = l == c->nlev - 1 ? 1 : n_states(c);
            W.st.assign(ns, nullptr);
            for (double *&q : W.st) {
                TRY(dalloc(c, &q, n));
                CUDA_TRY(c, cudaMemset(q, 0, n * sizeof(double)));
            }
        }
        c->un_ready = true;
    }
    while ((int)c->ck.size() < nck) {
        double *q = nullptr;
        TRY(dalloc(c, &q, c->L[0].n));
        c->ck.push_back(q);
    }
    return DMG_OK;
}

dmg_status copy_level(dmg_ctx *c, double *dst, const double *src, int l, cudaStream_t s) {
    return dcopy(c, dst, src, c->L[l].n, s);
}

dmg_status half64(dmg_ctx *c, int l, int color, cudaStream_t s) {
    Level &L = c->L[l];
    dmgk::k_smooth_half<double><<<grid_half(L.g), blk(), 0, s>>>(L.g, L.u, L.f, coef64(L), color, nullptr);
    return check_launch(c, "smooth");
}

// one forward V-cycle at level l on (u_l, f_l); save: keep the state after
// every half-sweep in un[l].st (and the coarsest solution in st[0])
dmg_status fwd_plain(dmg_ctx *c, int l, bool save, cudaStream_t s) {
    Level &L = c->L[l];
    ULevel &W = c->un[l];
    if (l == c->nlev - 1) {
        TRY(coarse_solve<double>(c, s));
        if (save) TRY(copy_level(c, W.st[0], L.u, l, s));
        return DMG_OK;
    }
    const int nu1 = c->p.nu1, nu2 = c->p.nu2, pf = c->p.symmetric ? 1 : 0;
    int h = 0;
    if (save && nu1 == 0) TRY(copy_level(c, W.st[n_states(c) - 1], L.u, l, s));
    for (int sw = 0; sw < nu1; sw++)
        for (int col = 0; col < 2; col++) {
            TRY(half64(c, l, col, s));
            if (save) TRY(copy_level(c, W.st[h], L.u, l, s));
            h++;
        }
    Level &C = c->L[l + 1];
    dmgk::k_residual<double><<<grid_int(L.g), blk(), 0, s>>>(L.g, L.u, L.f, coef64(L), L.r, nullptr);
    TRY(check_launch(c, "residual"));
    dmgk::k_restrict<double><<<grid_int(C.g), blk(), 0, s>>>(L.g, L.r, C.g, C.f, C.u, nullptr);
    TRY(check_launch(c, "restrict"));
    TRY(fwd_plain(c, l + 1, save, s));
    TRY(prolong<double>(c, l, s));
    for (int sw = 0; sw < nu2; sw++)
        for (int q = 0; q < 2; q++) {
            TRY(half64(c, l, q == 0 ? pf : 1 - pf, s));
            if (save) TRY(copy_level(c, W.st[h], L.u, l, s));
            h++;
        }
    return DMG_OK;
}

dmg_status rev_half(dmg_ctx *c, int l, int color, const double *U, cudaStream_t s) {
    Level &L = c->L[l];
    ULevel &W = c->un[l];
    dmgk::k_rev_other<<<grid_half(L.g), blk(), 0, s>>>(L.g, coef64(L), color, W.ub);
    TRY(check_launch(c, "rev_other"));
    dmgk::k_rev_own<<<grid_half(L.g), blk(), 0, s>>>(L.g, coef64(L), color, U, W.ub, W.fb, W.bx, W.by, W.bz,
                                                     W.mub);
    return check_launch(c, "rev_own");
}

// reverse of the V-cycle saved by fwd_plain(l, true): on entry un[l].ub is the
// cotangent of u_l after the cycle; on return it is the cotangent of u_l before
// it, un[l].fb has gained the cotangent of f_l, and the coefficient cotangents
// of levels l.. have gained the cycle's terms
dmg_status rev_plain(dmg_ctx *c, int l, cudaStream_t s) {
    Level &L = c->L[l];
    ULevel &W = c->un[l];
    if (l == c->nlev - 1) {
        // fbar += A^{-1} ubar (the inverse is symmetric); coefficient terms with the solution
        CUDA_TRY(c, cudaMemsetAsync(W.tmp, 0, L.n * sizeof(double), s));
        const int threads = c->nc < 32 ? 32 : (c->nc > 512 ? 512 : ((c->nc + 31) / 32) * 32);
        dmgk::k_coarse_solve<double><<<c->nb, threads, c->nc * sizeof(double), s>>>(L.g, c->Ainv, c->nc, W.ub,
                                                                                   W.tmp, nullptr);
        TRY(check_launch(c, "coarse_solve"));
        dmgk::k_rev_faces<<<grid_all(L.g), blk(), 0, s>>>(L.g, W.tmp, W.st[0], W.bx, W.by, W.bz, W.mub);
        TRY(check_launch(c, "rev_faces"));
        dmgk::k_add_interior<<<grid_int(L.g), blk(), 0, s>>>(L.g, W.tmp, W.fb);
        return check_launch(c, "add");
    }
    const int nu1 = c->p.nu1, nu2 = c->p.nu2, pf = c->p.symmetric ? 1 : 0;
    int h = 2 * (nu1 + nu2) - 1;
    for (int sw = nu2 - 1; sw >= 0; sw--)
        for (int q = 1; q >= 0; q--) {
            TRY(rev_half(c, l, q == 0 ? pf : 1 - pf, W.st[h], s));
            h--;
        }
    Level &C = c->L[l + 1];
    ULevel &WC = c->un[l + 1];
    dmgk::k_prolong_T<<<grid_all(C.g), blk(), 0, s>>>(L.g, W.ub, C.g, WC.ub);
    TRY(check_launch(c, "prolong_T"));
    CUDA_TRY(c, cudaMemsetAsync(WC.fb, 0, C.n * sizeof(double), s));
    TRY(rev_plain(c, l + 1, s));
    // defect r = f - A u after pre-smoothing; its cotangent is R^T fbar_{l+1}
    dmgk::k_restrict_T<<<grid_all(L.g), blk(), 0, s>>>(C.g, WC.fb, L.g, W.tmp);
    TRY(check_launch(c, "restrict_T"));
    dmgk::k_rev_defect<<<grid_int(L.g), blk(), 0, s>>>(L.g, coef64(L), W.tmp, W.ub, W.fb);
    TRY(check_launch(c, "rev_defect"));
    const double *Upre = nu1 > 0 ? W.st[2 * nu1 - 1] : W.st[n_states(c) - 1];
    dmgk::k_rev_faces<<<grid_all(L.g), blk(), 0, s>>>(L.g, W.tmp, Upre, W.bx, W.by, W.bz, W.mub);
    TRY(check_launch(c, "rev_faces"));
    for (int sw = nu1 - 1; sw >= 0; sw--)
        for (int col = 1; col >= 0; col--) {
            TRY(rev_half(c, l, col, W.st[h], s));
            h--;
        }
    return DMG_OK;
}

dmg_status vjp_unrolled_impl(dmg_ctx *c, const double *q, const double *w, int m, int stride, double *u,
                             double *qbar, double *Dbar, double *mubar, cudaStream_t s) {
    if (c->dim == 2) return fail(c, DMG_EINVAL, "dmg_vjp_unrolled is 3D only");
    TRY(need_whole(c));
    if (!q || !w) return fail(c, DMG_EINVAL, "q and w must not be NULL");
    if (m < 1 || m > 100000) return fail(c, DMG_EINVAL, "m must be in [1, 100000]");
    if (stride < 0) return fail(c, DMG_EINVAL, "stride must be >= 0");
    if (stride == 0) stride = std::max(1, (int)std::ceil(std::sqrt((double)m)));
    const int nck = (m + stride - 1) / stride;
    TRY(unrolled_alloc(c, nck));
    c->mask = nullptr;
    Level &L0 = c->L[0];
    ULevel &W0 = c->un[0];
    TRY(stage_in(c, q, L0.f, false, s));
    CUDA_TRY(c, cudaMemsetAsync(L0.u, 0, L0.n * sizeof(double), s));
    for (int cyc = 0; cyc < m; cyc++) {
        if (cyc % stride == 0) TRY(copy_level(c, c->ck[cyc / stride], L0.u, 0, s));
        TRY(fwd_plain(c, 0, false, s));
    }
    if (u) TRY(stage_out(c, L0.u, u, s));
    for (int l = 0; l < c->nlev; l++) {
        ULevel &W = c->un[l];
        for (double *x : {W.fb, W.bx, W.by, W.bz, W.mub})
            CUDA_TRY(c, cudaMemsetAsync(x, 0, c->L[l].n * sizeof(double), s));
    }
    TRY(stage_in(c, w, W0.ub, true, s));
    for (int cyc = m - 1; cyc >= 0; cyc--) {
        const int base = (cyc / stride) * stride;
        TRY(copy_level(c, L0.u, c->ck[cyc / stride], 0, s));
        for (int r = base; r < cyc; r++) TRY(fwd_plain(c, 0, false, s));
        TRY(fwd_plain(c, 0, true, s));
        TRY(rev_plain(c, 0, s));
    }
    if (qbar) TRY(stage_out(c, W0.fb, qbar, s));
    if (Dbar || mubar) {
        const int harm = c->p.face_mean == DMG_FACE_HARMONIC;
        for (int l = 0; l < c->nlev; l++) {
            Level &L = c->L[l];
            ULevel &W = c->un[l];
            dmgk::k_faces_to_vertex<<<grid_all(L.g), blk(), 0, s>>>(L.g, L.D, 1.0 / (L.h * L.h), harm, W.bx, W.by,
                                                                    W.bz, W.Db);
            TRY(check_launch(c, "faces_to_vertex"));
        }
        const int inj = c->p.coarsen == DMG_COARSEN_INJECTION;
        for (int l = c->nlev - 2; l >= 0; l--) {
            Level &L = c->L[l], &C = c->L[l + 1];
            dmgk::k_coarsen_T<<<grid_all(L.g), blk(), 0, s>>>(C.g, c->un[l + 1].Db, L.g, c->un[l].Db, inj);
            TRY(check_launch(c, "coarsen_T"));
            dmgk::k_coarsen_T<<<grid_all(L.g), blk(), 0, s>>>(C.g, c->un[l + 1].mub, L.g, c->un[l].mub, inj);
            TRY(check_launch(c, "coarsen_T"));
        }
        if (Dbar) TRY(stage_out(c, W0.Db, Dbar, s));
        if (mubar) TRY(stage_out(c, W0.mub, mubar, s));
    }
    return end_call(c, s);
}

// an NVTX range around one API call (visible in ncu / nsys timelines)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

#ifdef DMG_BOUNDS_CHECK
// checked builds: accesses counted outside their arrays since the last call
unsigned long long oob_delta() {
    static unsigned long long seen = 0;
    unsigned long long n = 0;
    if (cudaMemcpyFromSymbol(&n, dmgk::dmg_oob_count, sizeof(n)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const unsigned long long d = n - seen;
    seen = n;
    return d;
}
#endif

template <class F>
dmg_status guarded(dmg_ctx *c, F fn, const char *name = "dmg") {
    if (!c) return DMG_EINVAL;
    Range r(name);
    c->err[0] = 0;
    dmg_status st = fn();
#ifdef DMG_BOUNDS_CHECK
    cudaDeviceSynchronize();
    if (const unsigned long long d = oob_delta())
        return fail(c, DMG_ECUDA, "%s: %llu accesses outside their arrays", name, d);
#endif
    return st;
}

dmg_status destroy_impl(dmg_ctx *c) {
    if (!c) return DMG_OK;
    if (c->twin) destroy_impl(c->twin);
    if (c->twin_s) {
        cudaStreamSynchronize(c->twin_s);
        cudaStreamDestroy(c->twin_s);
    }
    if (c->ev_twin) cudaEventDestroy(c->ev_twin);
    if (c->lead_s) {
        cudaStreamSynchronize(c->lead_s);
        cudaStreamDestroy(c->lead_s);
    }
    if (c->ev_lead) cudaEventDestroy(c->ev_lead);
    if (c->cap_stream) cudaStreamSynchronize(c->cap_stream);
    graphs_reset(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    for (cudaStream_t st : {c->up, c->down})
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    for (int b = 0; b < 2; b++)
        for (cudaEvent_t e : {c->ev_in[b], c->ev_used[b], c->ev_ready_u[b], c->ev_ready[b], c->ev_out[b],
                              c->ev_in_q[b], c->ev_used_w[b], c->ev_qb[b]})
            if (e) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_aux) cudaEventDestroy(c->ev_aux);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    for (void *q : c->dev_allocs) cudaFree(q);
    if (c->hred) cudaFreeHost(c->hred);
    if (c->hact) cudaFreeHost(c->hact);
    if (c->hstatus) cudaFreeHost(c->hstatus);
    if (c->hact_a) cudaFreeHost(c->hact_a);
    delete c;
    return DMG_OK;
}

}  // namespace

// results of the arithmetic-rate probe land here only if they are impossible
__device__ double g_fma_sink64;
__device__ float g_fma_sink32;

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
    p->inner_cycles = 3;
    p->batch = 1;
    p->twin_adjoint = 1;
}

dmg_status dmg_setup(const dmg_params *p, const double *D, const double *mu, void *stream, dmg_ctx **out) {
    if (!out) return DMG_EINVAL;
    Range r("dmg_setup");
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

dmg_status dmg_setup_pyramid(const dmg_params *p, const int *slots_per_level, int nlevels, void *stream,
                             dmg_ctx **out) {
    if (!out) return DMG_EINVAL;
    Range r("dmg_setup_pyramid");
    *out = nullptr;
    if (!slots_per_level) {
        snprintf(g_setup_err, sizeof(g_setup_err), "slots_per_level must not be NULL");
        return DMG_EINVAL;
    }
    dmg_ctx *c = new (std::nothrow) dmg_ctx();
    if (!c) return DMG_ENOMEM;
    dmg_status st = setup_impl(c, p, nullptr, nullptr, S(stream), slots_per_level, nlevels);
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
        TRY(need_whole(c));
        if (!q || !u) return fail(c, DMG_EINVAL, "q and u must not be NULL");
        info_reset(info);
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        TRY(stage_in(c, q, l.f, false, s));
        dmg_status st = iterate(c, false, c->p.fixed_cycles, info, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return st;
        TRY(stage_out(c, l.u, u, s));
        TRY(end_call(c, s));
        return st;
    }, "dmg_solve");
}

dmg_status dmg_jvp(dmg_ctx *c, const double *u, const double *dq, const double *dD, const double *dmu,
                   double *du, dmg_info *info, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        TRY(need_whole(c));
        if (!du) return fail(c, DMG_EINVAL, "du must not be NULL");
        if ((dD || dmu) && !u) return fail(c, DMG_EINVAL, "u is needed for a D or mu tangent");
        info_reset(info);
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        if (dq) {
            TRY(stage_in(c, dq, l.f, false, s));
        } else {
            CUDA_TRY(c, cudaMemsetAsync(l.f, 0, l.n * sizeof(double), s));
        }
        if (dD || dmu) {
            TRY(stage_in(c, u, c->U0, true, s));
            if (dD) TRY(stage_in(c, dD, c->T1, false, s));
            if (dmu) TRY(stage_in(c, dmu, c->T2, false, s));
            double ih2 = 1.0 / (l.h * l.h);
            if (c->dim == 2)
                dmgk::k_dA2<<<grid_int2(l.g), blk(), 0, s>>>(l.g, c->U0, dD ? c->T1 : nullptr, dmu ? c->T2 : nullptr,
                                                             l.D, ih2, c->p.face_mean == DMG_FACE_HARMONIC, l.f);
            else
                dmgk::k_dA<<<grid_int(l.g), blk(), 0, s>>>(l.g, c->U0, dD ? c->T1 : nullptr, dmu ? c->T2 : nullptr,
                                                           l.D, ih2, c->p.face_mean == DMG_FACE_HARMONIC, l.f);
            TRY(check_launch(c, "dA"));
        }
        dmg_status st = iterate(c, false, c->p.fixed_cycles, info, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return st;
        TRY(stage_out(c, l.u, du, s));
        TRY(end_call(c, s));
        return st;
    }, "dmg_jvp");
}

dmg_status dmg_solve_vjp(dmg_ctx *c, const double *q, const double *w, double *u, double *qbar, double *Dbar,
                         double *mubar, dmg_info *info_fwd, dmg_info *info_adj, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        TRY(need_whole(c));
        if (!q || !w) return fail(c, DMG_EINVAL, "q and w must not be NULL");
        info_reset(info_fwd);
        info_reset(info_adj);
        cudaStream_t s = S(stream);
        if (c->p.twin_adjoint) {
            // without device memory for the twin the pair runs in one lane
            const dmg_status tw = twin_ready(c, s);
            if (tw == DMG_OK) return solve_vjp_twin(c, q, w, u, qbar, Dbar, mubar, info_fwd, info_adj, s);
            if (tw != DMG_ENOMEM) return tw;
            c->err[0] = 0;
        }
        Level &l = c->L[0];
        // w goes to T3 on the side stream while the forward iterates
        CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));
        CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        TRY(stage_in(c, w, c->T3, false, c->side, -1, c->stage2));
        CUDA_TRY(c, cudaEventRecord(c->ev_aux, c->side));
        TRY(stage_in(c, q, l.f, false, s));
        dmg_status st = iterate(c, false, c->p.fixed_cycles, info_fwd, s);
        if (st != DMG_OK && st != DMG_ENOCONV) {
            cudaStreamSynchronize(c->side);
            return st;
        }
        // the forward solution stays on the device for the gradient; its read-out
        // (side stream) overlaps the adjoint iteration
        TRY(dcopy(c, c->U0, l.u, l.n, s));
        CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_aux, 0));
        TRY(dcopy(c, l.f, c->T3, l.n, s));
        if (u) {
            CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));
            CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
            TRY(stage_out(c, c->U0, u, c->side, -1, c->stage2));
        }
        dmg_status st2 = iterate(c, true, 0, info_adj, s);
        if (st2 != DMG_OK && st2 != DMG_ENOCONV) {
            cudaStreamSynchronize(c->side);
            return st2;
        }
        if (qbar) {   // overlaps the gradient kernel
            CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));
            CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
            TRY(stage_out(c, l.u, qbar, c->side, -1, c->stage2));
        }
        CUDA_TRY(c, cudaEventRecord(c->ev_join, c->side));
        if (Dbar || mubar) TRY(grad_out(c, c->U0, l.u, Dbar, mubar, s));
        CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_join, 0));
        TRY(end_call(c, s));
        return st != DMG_OK ? st : st2;
    }, "dmg_solve_vjp");
}

dmg_status dmg_solve_vjp_many(dmg_ctx *c, int npairs, const double *const *q, const double *const *w,
                              double *const *u, double *const *qbar, double *const *Dbar, double *const *mubar,
                              dmg_info *info_fwd, dmg_info *info_adj, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        TRY(need_whole(c));
        if (info_fwd) for (int i = 0; i < npairs; i++) info_reset(info_fwd + i);
        if (info_adj) for (int i = 0; i < npairs; i++) info_reset(info_adj + i);
        return solve_vjp_many_impl(c, npairs, q, w, u, qbar, Dbar, mubar, info_fwd, info_adj, S(stream));
    }, "dmg_solve_vjp_many");
}

dmg_status dmg_vjp(dmg_ctx *c, const double *u, const double *w, int cycles, double *qbar, double *Dbar,
                   double *mubar, dmg_info *info, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        TRY(need_whole(c));
        if (!w) return fail(c, DMG_EINVAL, "w must not be NULL");
        if ((Dbar || mubar) && !u) return fail(c, DMG_EINVAL, "u is needed for Dbar / mubar");
        if (cycles < 0) return fail(c, DMG_EINVAL, "cycles must be >= 0");
        info_reset(info);
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        // u is needed only by the gradient kernel at the end: its transfer and
        // gather run on the side stream while the adjoint iterates
        const bool need_u = Dbar || mubar;
        if (need_u) {
            CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));
            CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
            TRY(stage_in(c, u, c->U0, true, c->side, -1, c->stage2));
            CUDA_TRY(c, cudaEventRecord(c->ev_join, c->side));
        }
        TRY(stage_in(c, w, l.f, false, s));
        dmg_status st = iterate(c, true, cycles, info, s);
        if (st != DMG_OK && st != DMG_ENOCONV) {
            if (need_u) cudaStreamSynchronize(c->side);
            return st;
        }
        if (need_u) CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_join, 0));
        if (qbar && need_u) {
            // qbar's read-out on the side stream overlaps the gradient kernel
            CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));
            CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
            TRY(stage_out(c, l.u, qbar, c->side, -1, c->stage2));
            CUDA_TRY(c, cudaEventRecord(c->ev_join, c->side));
        } else if (qbar) {
            TRY(stage_out(c, l.u, qbar, s));
        }
        if (Dbar || mubar) {
            TRY(grad_out(c, c->U0, l.u, Dbar, mubar, s));
            if (qbar) CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_join, 0));
        }
        TRY(end_call(c, s));
        return st;
    }, "dmg_vjp");
}

}  // extern "C"

namespace {

// first kept index per axis: the smallest m with m h >= edge (1 - 1e-12)
dmg_status margins(dmg_ctx *c, double edge, dmgk::Margins *m) {
    if (c->dim == 2) return fail(c, DMG_EINVAL, "the response operator is 3D only");
    if (!(edge >= 0.0) || !std::isfinite(edge)) return fail(c, DMG_EINVAL, "edge must be finite and >= 0");
    const double h = c->p.h, e = edge * (1.0 - 1e-12);
    auto first = [&](int n) {
        long long k = (long long)std::ceil(e / h);
        if (k < 0) k = 0;
        return (int)std::min<long long>(k, n);
    };
    m->x = first(c->p.nx);
    m->y = first(c->p.ny);
    m->z = first(c->p.nz);
    return DMG_OK;
}

}  // namespace

extern "C" {

dmg_status dmg_response(dmg_ctx *c, const double *q, double edge, double *Le, double *u, dmg_info *info,
                        void *stream) {
    return guarded(c, [&]() -> dmg_status {
        TRY(need_whole(c));
        if (!q || !Le) return fail(c, DMG_EINVAL, "q and Le must not be NULL");
        dmgk::Margins m;
        TRY(margins(c, edge, &m));
        info_reset(info);
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        TRY(stage_in(c, q, l.f, false, s));
        dmg_status st = iterate(c, false, c->p.fixed_cycles, info, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return st;
        if (u) TRY(stage_out(c, l.u, u, s));
        dmgk::k_response<<<grid_all(l.g), blk(), 0, s>>>(l.g, m, l.mu, l.u, nullptr, nullptr, c->T3);
        TRY(check_launch(c, "response"));
        TRY(stage_out(c, c->T3, Le, s));
        TRY(end_call(c, s));
        return st;
    }, "dmg_response");
}

dmg_status dmg_response_jvp(dmg_ctx *c, const double *u, const double *dq, const double *dD, const double *dmu,
                            double edge, double *dLe, dmg_info *info, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        TRY(need_whole(c));
        if (!u || !dLe) return fail(c, DMG_EINVAL, "u and dLe must not be NULL");
        dmgk::Margins m;
        TRY(margins(c, edge, &m));
        info_reset(info);
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        if (dq) {
            TRY(stage_in(c, dq, l.f, false, s));
        } else {
            CUDA_TRY(c, cudaMemsetAsync(l.f, 0, l.n * sizeof(double), s));
        }
        TRY(stage_in(c, u, c->U0, true, s));
        if (dD) TRY(stage_in(c, dD, c->T1, false, s));
        if (dmu) TRY(stage_in(c, dmu, c->T2, false, s));
        if (dD || dmu) {
            const double ih2 = 1.0 / (l.h * l.h);
            dmgk::k_dA<<<grid_int(l.g), blk(), 0, s>>>(l.g, c->U0, dD ? c->T1 : nullptr, dmu ? c->T2 : nullptr,
                                                       l.D, ih2, c->p.face_mean == DMG_FACE_HARMONIC, l.f);
            TRY(check_launch(c, "dA"));
        }
        dmg_status st = iterate(c, false, c->p.fixed_cycles, info, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return st;
        // dLe = M(mu du + dmu u)
        dmgk::k_response<<<grid_all(l.g), blk(), 0, s>>>(l.g, m, l.mu, l.u, dmu ? c->T2 : nullptr, c->U0, c->T3);
        TRY(check_launch(c, "response"));
        TRY(stage_out(c, c->T3, dLe, s));
        TRY(end_call(c, s));
        return st;
    }, "dmg_response_jvp");
}

dmg_status dmg_response_vjp(dmg_ctx *c, const double *u, const double *rbar, double edge, double *qbar,
                            double *Dbar, double *mubar, dmg_info *info, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        TRY(need_whole(c));
        if (!rbar) return fail(c, DMG_EINVAL, "rbar must not be NULL");
        if ((Dbar || mubar) && !u) return fail(c, DMG_EINVAL, "u is needed for Dbar / mubar");
        dmgk::Margins m;
        TRY(margins(c, edge, &m));
        info_reset(info);
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        TRY(stage_in(c, rbar, c->T3, false, s));
        dmgk::k_response_cot<<<grid_all(l.g), blk(), 0, s>>>(l.g, m, l.mu, c->T3, l.f);
        TRY(check_launch(c, "response_cot"));
        dmg_status st = iterate(c, true, 0, info, s);
        if (st != DMG_OK && st != DMG_ENOCONV) return st;
        if (qbar) TRY(stage_out(c, l.u, qbar, s));
        if (Dbar || mubar) {
            TRY(stage_in(c, u, c->U0, true, s));
            const double ih2 = 1.0 / (l.h * l.h);
            launch_grad(s, l.g, c->U0, l.u, l.D, ih2,
                                                         c->p.face_mean == DMG_FACE_HARMONIC, Dbar ? c->T1 : nullptr,
                                                         c->T2);
            TRY(check_launch(c, "grad"));
            if (mubar) {
                dmgk::k_response_mubar<<<grid_all(l.g), blk(), 0, s>>>(l.g, m, c->U0, c->T3, c->T2);
                TRY(check_launch(c, "response_mubar"));
            }
            if (Dbar) TRY(stage_out(c, c->T1, Dbar, s));
            if (mubar) TRY(stage_out(c, c->T2, mubar, s));
        }
        TRY(end_call(c, s));
        return st;
    }, "dmg_response_vjp");
}

dmg_status dmg_residual(dmg_ctx *c, const double *q, const double *u, double *out, void *stream) {
    return guarded(c, [&]() -> dmg_status {
        if (!q || !u || !out) return fail(c, DMG_EINVAL, "q, u and out must not be NULL");
        if (c->pyramid) return fail(c, DMG_EINVAL, "a pyramid pool serves its slots only (dmg_slot_* calls)");
        cudaStream_t s = S(stream);
        Level &l = c->L[0];
        TRY(stage_in(c, q, c->T3, false, s));
        TRY(stage_in(c, u, c->U0, true, s));
        TRY(resid_norm_async(c, c->U0, c->T3, nullptr, 0, nullptr, s));
        TRY(norm2_async(c, c->T3, 1, s));
        TRY(finish_reduce(c, s));
        (void)l;
        for (int b = 0; b < c->nb; b++) {
            out[2 * b] = std::sqrt(hred(c, b, 0));
            out[2 * b + 1] = std::sqrt(hred(c, b, 1));
        }
        return DMG_OK;
    }, "dmg_residual");
}

dmg_status dmg_destroy(dmg_ctx *c) { return destroy_impl(c); }

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

dmg_status dmg_vjp_unrolled(dmg_ctx *c, const double *q, const double *w, int m, int stride, double *u,
                            double *qbar, double *Dbar, double *mubar, void *stream) {
    return guarded(c, [&]() { return vjp_unrolled_impl(c, q, w, m, stride, u, qbar, Dbar, mubar, S(stream)); }, "dmg_vjp_unrolled");
}

dmg_status dmg_slot_load(dmg_ctx *c, int slot, const double *D, const double *mu, void *stream) {
    return guarded(c, [&]() { return slot_load_impl(c, slot, D, mu, S(stream)); }, "dmg_slot_load");
}

dmg_status dmg_set_coefficients(dmg_ctx *c, const double *D, const double *mu, void *stream) {
    return guarded(c, [&]() { return set_coefficients_impl(c, D, mu, S(stream)); }, "dmg_set_coefficients");
}

dmg_status dmg_probe_fma(int fp64, double *fma_per_s, void *stream) {
    Range r("dmg_probe_fma");
    if (!fma_per_s) return DMG_EINVAL;
    *fma_per_s = 0.0;
    cudaStream_t s = S(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return DMG_ECUDA;
    void *sink = nullptr;
    if ((fp64 ? cudaGetSymbolAddress(&sink, g_fma_sink64) : cudaGetSymbolAddress(&sink, g_fma_sink32)) !=
        cudaSuccess)
        return DMG_ECUDA;
    // 8 blocks of 256 threads per SM (one full wave); about 20 ms of work at the expected rate
    const int blocks = 8 * sms, threads = 256;
    const int iters = fp64 ? 2048 : 65536;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    dmg_status st = DMG_OK;
    float ms = 0.0f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = DMG_ECUDA;
    for (int rep = 0; rep < 3 && st == DMG_OK; rep++) {   // the first launch warms up
        if (cudaEventRecord(e0, s) != cudaSuccess) st = DMG_ECUDA;
        if (fp64)
            dmgk::k_fma_probe<double><<<blocks, threads, 0, s>>>(iters, (double *)sink);
        else
            dmgk::k_fma_probe<float><<<blocks, threads, 0, s>>>(iters, (float *)sink);
        if (st == DMG_OK && (cudaPeekAtLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = DMG_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != DMG_OK || ms <= 0.0f) return DMG_ECUDA;
    *fma_per_s = (double)blocks * threads * dmgk::kFmaChains * iters / (ms * 1e-3);
    return DMG_OK;
}

dmg_status dmg_slot_begin(dmg_ctx *c, int slot, int phase, const double *a, const double *b, const double *d,
                          void *stream) {
    return guarded(c, [&]() { return slot_begin_impl(c, slot, phase, a, b, d, S(stream)); }, "dmg_slot_begin");
}

dmg_status dmg_step_launch(dmg_ctx *c, void *stream) {
    return guarded(c, [&]() { return step_launch_impl(c, S(stream)); }, "dmg_step_launch");
}

dmg_status dmg_step_finish(dmg_ctx *c, void *stream, int *ended, int *nended) {
    return guarded(c, [&]() { return step_finish_impl(c, S(stream), ended, nended); }, "dmg_step_finish");
}

dmg_status dmg_slot_result(const dmg_ctx *c, int slot, int *status, int *cycles, double *rel) {
    if (!c || slot < 0 || slot >= c->nb) return DMG_EINVAL;
    const Slot &sl = c->slots[slot];
    if (status) *status = slot_busy(sl) ? -1 : (sl.phase < 0 ? DMG_OK : sl.status);
    if (cycles) *cycles = sl.steps * (c->p.precision == DMG_MIXED ? c->p.inner_cycles : 1);
    if (rel) *rel = sl.rel;
    return DMG_OK;
}

dmg_status dmg_slot_read(dmg_ctx *c, int slot, double *u, double *x, double *Dbar, double *mubar, void *stream) {
    return guarded(c, [&]() { return slot_read_impl(c, slot, u, x, Dbar, mubar, S(stream)); }, "dmg_slot_read");
}

size_t dmg_device_bytes(const dmg_ctx *c) { return c ? c->dev_bytes + (c->twin ? c->twin->dev_bytes : 0) : 0; }

void dmg_debug_fail_alloc(long long n) { g_fail_alloc_at.store(n > 0 ? n : 0); }

void dmg_debug_grad_per_vertex(int on) { g_grad_per_vertex.store(on ? 1 : 0); }

long long dmg_debug_oob_count(void) {
#ifdef DMG_BOUNDS_CHECK
    unsigned long long n = 0;
    if (cudaMemcpyFromSymbol(&n, dmgk::dmg_oob_count, sizeof(n)) != cudaSuccess) {
        cudaGetLastError();
        return -2;
    }
    return (long long)n;
#else
    return -1;
#endif
}

dmg_status dmg_batch_info(const dmg_ctx *c, int *cycles, double *rel) {
    if (!c) return DMG_EINVAL;
    for (int b = 0; b < c->nb; b++) {
        if (cycles) cycles[b] = c->bcyc[b];
        if (rel) rel[b] = c->brel[b];
    }
    return DMG_OK;
}

int dmg_levels(const dmg_ctx *c) { return c ? c->nlev : 0; }

dmg_status dmg_tile(const dmg_ctx *c, int level, int fp32, int *bx, int *by) {
    if (!c || level < 0 || level >= c->nlev) return DMG_EINVAL;
    const dim3 b = c->tb[fp32 ? 1 : 0][level];
    if (bx) *bx = (int)b.x;
    if (by) *by = (int)b.y;
    return DMG_OK;
}

dmg_status dmg_level_shape(const dmg_ctx *c, int level, int *nx, int *ny, int *nz) {
    if (!c || level < 0 || level >= c->nlev) return DMG_EINVAL;
    if (nx) *nx = c->L[level].g.nx;
    if (ny) *ny = c->L[level].g.ny;
    if (nz) *nz = c->L[level].g.nz;
    return DMG_OK;
}

unsigned long long dmg_launch_count(const dmg_ctx *c) {
    return c ? c->launches + (c->twin ? c->twin->launches : 0) : 0;
}

dmg_status dmg_profile_begin(dmg_ctx *c, int kernel, int level, int precision_fp32, int max_launches) {
    if (!c || max_launches < 1 || level < 0 || level >= c->nlev) return DMG_EINVAL;
    CUDA_TRY(c, cudaDeviceSynchronize());
    graphs_reset(c);   // graphs are re-captured with event nodes
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.assign(2 * (size_t)max_launches, nullptr);
    c->prof_n.assign((size_t)max_launches, 0);
    c->prof_open = -1;
    for (auto &e : c->prof_ev) CUDA_TRY(c, cudaEventCreate(&e));
    c->prof_free.clear();
    for (int i = max_launches - 1; i >= 0; i--) c->prof_free.push_back(i);
    c->prof_direct.clear();
    c->prof_kernel = kernel;
    c->prof_level = level;
    c->prof_fp32 = precision_fp32 ? 1 : 0;
    c->prof_count = 0;
    c->prof_ms = 0.0;
    return DMG_OK;
}

dmg_status dmg_profile_end(dmg_ctx *c, long long *launches, double *total_ms) {
    if (!c) return DMG_EINVAL;
    CUDA_TRY(c, cudaDeviceSynchronize());
    prof_harvest(c, c->prof_direct, true);
    if (launches) *launches = c->prof_count;
    if (total_ms) *total_ms = c->prof_ms;
    c->prof_kernel = -1;
    graphs_reset(c);   // drop the event nodes
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof_free.clear();
    c->prof_count = 0;
    c->prof_ms = 0.0;
    return DMG_OK;
}

}  // extern "C"
