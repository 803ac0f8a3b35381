// Device kernels of the B300 multigrid solver for -div(D grad u) + mu u = q
// (arXiv 2608.00760, Eq. 1), templated on the arithmetic type (double for the
// FP64 path, float for the inner V-cycles of mixed-precision refinement).
//
// Layout: every field is a padded C-order array [nz][ny][sy] (sy >= nx, a
// multiple of 32 elements, so every row starts on a 256-byte boundary in FP64);
// element (i, j, k) is at k*sz + j*sy + i with sz = ny*sy. Values on boundary
// vertices of u, f and r are zero and no kernel writes them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmgk {

struct Geom {
    int nx, ny, nz;   // vertices per axis, boundary included
    int sy;           // row pitch in elements
    long long sz;     // plane pitch in elements
    __host__ __device__ __forceinline__ long long at(int i, int j, int k) const {
        return (long long)k * sz + (long long)j * sy + i;
    }
};

// ---------------------------------------------------------------------------
// Coefficient access. The 7-point operator (Eq. 1, second-order differences)
//   (A u)_p = sum_{j in nbr(p)} a_pj (u_p - u_j) + mu_p u_p,  a_pj = face(D_p, D_j) / h^2
// is read either from precomputed faces (FP64: the couplings a and 1/diag are
// stored, which keeps the FP64 ALU work per point at 6 FMA + 1 MUL) or from
// vertex values (FP32: the faces are formed on the fly, which halves the bytes
// of this memory-bound path).

template <class T>
struct FaceCoef {
    const T *cx, *cy, *cz;   // a between p and p+x, p+y, p+z
    const T *diag, *invd;    // diagonal and its reciprocal (0 on the boundary)
    __device__ __forceinline__ void couplings(long long p, int sy, long long sz, T a[6]) const {
        a[0] = __ldg(cx + p - 1);  a[1] = __ldg(cx + p);
        a[2] = __ldg(cy + p - sy); a[3] = __ldg(cy + p);
        a[4] = __ldg(cz + p - sz); a[5] = __ldg(cz + p);
    }
    __device__ __forceinline__ T get_diag(long long p, const T *) const { return __ldg(diag + p); }
    __device__ __forceinline__ T inv_diag(long long p, const T *) const { return __ldg(invd + p); }
};

// Dh = D / (2 h^2) for the arithmetic face mean (face = Dh_p + Dh_j),
// Dh = D / h^2 for the harmonic mean (face = 2 Dh_p Dh_j / (Dh_p + Dh_j)).
template <class T, bool HARM>
struct VertCoef {
    const T *Dh, *mu;
    __device__ __forceinline__ static T face(T a, T b) {
        if (HARM) return T(2) * a * b / (a + b);
        return a + b;
    }
    __device__ __forceinline__ void couplings(long long p, int sy, long long sz, T a[6]) const {
        T d = __ldg(Dh + p);
        a[0] = face(d, __ldg(Dh + p - 1));  a[1] = face(d, __ldg(Dh + p + 1));
        a[2] = face(d, __ldg(Dh + p - sy)); a[3] = face(d, __ldg(Dh + p + sy));
        a[4] = face(d, __ldg(Dh + p - sz)); a[5] = face(d, __ldg(Dh + p + sz));
    }
    __device__ __forceinline__ T get_diag(long long p, const T *a) const {
        return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + __ldg(mu + p));
    }
    __device__ __forceinline__ T inv_diag(long long p, const T *a) const {
        return T(1) / get_diag(p, a);
    }
};

// ---------------------------------------------------------------------------
// Red-Black Gauss-Seidel half-sweep (Eq. 9): every interior vertex of colour
// (i+j+k) mod 2 == color takes u_p = (f_p + sum_j a_pj u_j) / diag_p. Vertices
// of one colour are not coupled, so the update is in place and race-free.
// Thread layout: x covers the vertices of the colour in a row (every other i).
template <class T, class C>
__global__ void __launch_bounds__(256) k_smooth_half(Geom g, T *__restrict__ u,
                                                     const T *__restrict__ f, C c, int color) {
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (j > g.ny - 2) return;
    int i = 1 + ((1 + j + k + color) & 1) + 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i > g.nx - 2) return;
    long long p = g.at(i, j, k);
    T a[6];
    c.couplings(p, g.sy, g.sz, a);
    T s = __ldg(f + p);
    s = fma(a[0], u[p - 1], s);
    s = fma(a[1], u[p + 1], s);
    s = fma(a[2], u[p - g.sy], s);
    s = fma(a[3], u[p + g.sy], s);
    s = fma(a[4], u[p - g.sz], s);
    s = fma(a[5], u[p + g.sz], s);
    u[p] = s * c.inv_diag(p, a);
}

// residual value at an interior vertex: f_p - diag_p u_p + sum_j a_pj u_j
template <class T, class C>
__device__ __forceinline__ T residual_at(const Geom &g, const T *__restrict__ u,
                                         const T *__restrict__ f, const C &c, long long p) {
    T a[6];
    c.couplings(p, g.sy, g.sz, a);
    T s = fma(-c.get_diag(p, a), __ldg(u + p), __ldg(f + p));
    s = fma(a[0], __ldg(u + p - 1), s);
    s = fma(a[1], __ldg(u + p + 1), s);
    s = fma(a[2], __ldg(u + p - g.sy), s);
    s = fma(a[3], __ldg(u + p + g.sy), s);
    s = fma(a[4], __ldg(u + p - g.sz), s);
    s = fma(a[5], __ldg(u + p + g.sz), s);
    return s;
}

// r = f - A u on interior vertices (the defect, Eqs. 13-14)
template <class T, class C>
__global__ void __launch_bounds__(256) k_residual(Geom g, const T *__restrict__ u,
                                                  const T *__restrict__ f, C c, T *__restrict__ r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    long long p = g.at(i, j, k);
    r[p] = residual_at(g, u, f, c, p);
}

// Full-weighting restriction (Eq. 7, 1/4[1 2 1] per axis) of a fine field onto
// coarse interior vertices. The 27 fine points around 2I are all fine-interior.
template <class T>
__global__ void __launch_bounds__(256) k_restrict(Geom gf, const T *__restrict__ r, Geom gc,
                                                  T *__restrict__ fc) {
    int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int J = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int K = blockIdx.z + 1;
    if (I > gc.nx - 2 || J > gc.ny - 2) return;
    long long p = gf.at(2 * I, 2 * J, 2 * K);
    T s = T(0);
#pragma unroll
    for (int c = -1; c <= 1; c++) {
        T sp = T(0);
#pragma unroll
        for (int b = -1; b <= 1; b++) {
            long long q = p + c * gf.sz + b * gf.sy;
            T row = __ldg(r + q - 1) + T(2) * __ldg(r + q) + __ldg(r + q + 1);
            sp += (b == 0 ? T(2) : T(1)) * row;
        }
        s += (c == 0 ? T(2) : T(1)) * sp;
    }
    fc[gc.at(I, J, K)] = s * T(1.0 / 64.0);
}

// Prolongation I = 2^3 R^T (Eq. 17) and correction: u_fine += trilinear(e)
// on fine interior vertices. e is zero on the coarse boundary.
template <class T>
__global__ void __launch_bounds__(256) k_prolong_add(Geom gc, const T *__restrict__ e, Geom gf,
                                                     T *__restrict__ u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (i > gf.nx - 2 || j > gf.ny - 2) return;
    int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    int ni = (i & 1) + 1, nj = (j & 1) + 1, nk = (k & 1) + 1;
    T wi = (i & 1) ? T(0.5) : T(1), wj = (j & 1) ? T(0.5) : T(1), wk = (k & 1) ? T(0.5) : T(1);
    T s = T(0);
    for (int c = 0; c < nk; c++) {
        T sj = T(0);
        for (int b = 0; b < nj; b++) {
            long long q = gc.at(i0, j0 + b, k0 + c);
            T si = __ldg(e + q);
            if (ni == 2) si += __ldg(e + q + 1);
            sj += si;
        }
        s += sj;
    }
    long long p = gf.at(i, j, k);
    u[p] += (wi * wj * wk) * s;
}

// Exact coarsest-level solve u = A^{-1} f with the symmetric inverse built at
// setup; one block, one thread per coarsest interior unknown.
template <class T>
__global__ void k_coarse_solve(Geom g, const T *__restrict__ Ainv, int n, const T *__restrict__ f,
                               T *__restrict__ u) {
    extern __shared__ unsigned char smem_raw[];
    T *fs = reinterpret_cast<T *>(smem_raw);
    int nxi = g.nx - 2, nyi = g.ny - 2;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        int i = c % nxi + 1, j = (c / nxi) % nyi + 1, k = c / (nxi * nyi) + 1;
        fs[c] = f[g.at(i, j, k)];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        T s = T(0);
        for (int c = 0; c < n; c++) s = fma(Ainv[(long long)r * n + c], fs[c], s);
        int i = r % nxi + 1, j = (r / nxi) % nyi + 1, k = r / (nxi * nyi) + 1;
        u[g.at(i, j, k)] = s;
    }
}

// ---------------------------------------------------------------------------
// setup kernels

// Coefficient coarsening for the rediscretised coarse operator: full weighting
// on coarse interior vertices, injection on the coarse boundary (or injection
// everywhere). One thread per coarse vertex.
__global__ void k_coarsen(Geom gf, const double *__restrict__ X, Geom gc, double *__restrict__ Xc,
                          int inject) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    int J = blockIdx.y * blockDim.y + threadIdx.y;
    int K = blockIdx.z;
    if (I >= gc.nx || J >= gc.ny) return;
    long long p = gf.at(2 * I, 2 * J, 2 * K);
    bool interior = I > 0 && J > 0 && K > 0 && I < gc.nx - 1 && J < gc.ny - 1 && K < gc.nz - 1;
    double s;
    if (inject || !interior) {
        s = X[p];
    } else {
        s = 0.0;
        for (int c = -1; c <= 1; c++)
            for (int b = -1; b <= 1; b++)
                for (int a = -1; a <= 1; a++) {
                    double w = (a == 0 ? 0.5 : 0.25) * (b == 0 ? 0.5 : 0.25) * (c == 0 ? 0.5 : 0.25);
                    s += w * X[p + c * gf.sz + b * gf.sy + a];
                }
    }
    Xc[gc.at(I, J, K)] = s;
}

__device__ __forceinline__ double face_mean(double a, double b, int harm) {
    return harm ? 2.0 * a * b / (a + b) : 0.5 * (a + b);
}

// FP64 face couplings a = face(D_p, D_j)/h^2 (stored at the lower vertex of each
// face), diagonal and its reciprocal. One thread per vertex.
__global__ void k_build_faces(Geom g, const double *__restrict__ D, const double *__restrict__ mu,
                              double ih2, int harm, double *cx, double *cy, double *cz,
                              double *diag, double *invd) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    long long p = g.at(i, j, k);
    double d = D[p];
    cx[p] = i < g.nx - 1 ? face_mean(d, D[p + 1], harm) * ih2 : 0.0;
    cy[p] = j < g.ny - 1 ? face_mean(d, D[p + g.sy], harm) * ih2 : 0.0;
    cz[p] = k < g.nz - 1 ? face_mean(d, D[p + g.sz], harm) * ih2 : 0.0;
    bool interior = i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1;
    if (interior) {
        double s = face_mean(d, D[p - 1], harm) + face_mean(d, D[p + 1], harm) +
                   face_mean(d, D[p - g.sy], harm) + face_mean(d, D[p + g.sy], harm) +
                   face_mean(d, D[p - g.sz], harm) + face_mean(d, D[p + g.sz], harm);
        double dg = s * ih2 + mu[p];
        diag[p] = dg;
        invd[p] = 1.0 / dg;
    } else {
        diag[p] = 0.0;
        invd[p] = 0.0;
    }
}

// FP32 vertex coefficients for the inner V-cycles: Dh = D * scale, mu32 = mu.
__global__ void k_build_vertex32(Geom g, const double *__restrict__ D, const double *__restrict__ mu,
                                 double scale, float *Dh, float *mu32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    long long p = g.at(i, j, k);
    Dh[p] = (float)(D[p] * scale);
    mu32[p] = (float)mu[p];
}

// Dense coarsest matrix (n x n, interior unknowns in x-fastest order) from the
// FP64 faces; row-major into M with row stride 2n (the right half is set to I).
__global__ void k_coarse_assemble(Geom g, FaceCoef<double> c, int n, double *M) {
    int nxi = g.nx - 2, nyi = g.ny - 2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * 2 * n;
         t += (long long)gridDim.x * blockDim.x) {
        int r = (int)(t / (2 * n)), col = (int)(t % (2 * n));
        double v = 0.0;
        if (col >= n) {
            v = (col - n == r) ? 1.0 : 0.0;
        } else {
            int ri = r % nxi + 1, rj = (r / nxi) % nyi + 1, rk = r / (nxi * nyi) + 1;
            int ci = col % nxi + 1, cj = (col / nxi) % nyi + 1, ck = col / (nxi * nyi) + 1;
            long long p = g.at(ri, rj, rk);
            int di = ci - ri, dj = cj - rj, dk = ck - rk;
            if (di == 0 && dj == 0 && dk == 0) v = c.diag[p];
            else if (dj == 0 && dk == 0 && di == -1) v = -c.cx[p - 1];
            else if (dj == 0 && dk == 0 && di == 1) v = -c.cx[p];
            else if (di == 0 && dk == 0 && dj == -1) v = -c.cy[p - g.sy];
            else if (di == 0 && dk == 0 && dj == 1) v = -c.cy[p];
            else if (di == 0 && dj == 0 && dk == -1) v = -c.cz[p - g.sz];
            else if (di == 0 && dj == 0 && dk == 1) v = -c.cz[p];
        }
        M[t] = v;
    }
}

// In-block Gauss-Jordan inversion of the SPD matrix in [M | I] (no pivoting is
// needed for SPD). Writes the symmetrised inverse in FP64 and FP32 and sets
// *status = 1 if a pivot is not positive. One block; n <= 512.
__global__ void k_gauss_jordan(double *M, int n, double *Ainv, float *Ainv32, int *status) {
    __shared__ double colk[512];
    __shared__ double piv;
    __shared__ int bad;
    int n2 = 2 * n;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < n; k++) {
        if (threadIdx.x == 0) {
            piv = M[(long long)k * n2 + k];
            if (!(piv > 0.0)) bad = 1;
        }
        __syncthreads();
        if (bad) break;
        for (int c = threadIdx.x; c < n2; c += blockDim.x) M[(long long)k * n2 + c] /= piv;
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) colk[r] = M[(long long)r * n2 + k];
        __syncthreads();
        for (long long t = threadIdx.x; t < (long long)n * n2; t += blockDim.x) {
            int r = (int)(t / n2), c = (int)(t % n2);
            if (r != k) M[t] -= colk[r] * M[(long long)k * n2 + c];
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) *status = 1;
        return;
    }
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        int r = (int)(t / n), c = (int)(t % n);
        double v = 0.5 * (M[(long long)r * n2 + n + c] + M[(long long)c * n2 + n + r]);
        Ainv[t] = v;
        Ainv32[t] = (float)v;
    }
    if (threadIdx.x == 0) *status = 0;
}

// ---------------------------------------------------------------------------
// reductions (deterministic: fixed grid, fixed shuffle order, fixed final order)

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += sh[q];
    return s;  // valid in thread 0
}

// partial[b] = sum over this block's interior vertices of (f - A u)^2; optional
// outputs: r (same type) and r32 = (float)(r * r32_scale).
template <class T, class C>
__global__ void __launch_bounds__(256) k_resid_norm(Geom g, const T *__restrict__ u,
                                                    const T *__restrict__ f, C c,
                                                    T *__restrict__ rout, float *__restrict__ r32,
                                                    double r32_scale, double *partial) {
    __shared__ double sh[8];
    int nxi = g.nx - 2, nyi = g.ny - 2, nzi = g.nz - 2;
    unsigned total = (unsigned)nxi * nyi * nzi;
    double acc = 0.0;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        unsigned i = t % nxi, rest = t / nxi;
        unsigned j = rest % nyi, k = rest / nyi;
        long long p = g.at(i + 1, j + 1, k + 1);
        T r = residual_at(g, u, f, c, p);
        if (rout) rout[p] = r;
        if (r32) r32[p] = (float)((double)r * r32_scale);
        acc = fma((double)r, (double)r, acc);
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// partial[b] = sum over this block's interior vertices of x^2
__global__ void __launch_bounds__(256) k_norm2(Geom g, const double *__restrict__ x, double *partial) {
    __shared__ double sh[8];
    int nxi = g.nx - 2, nyi = g.ny - 2, nzi = g.nz - 2;
    unsigned total = (unsigned)nxi * nyi * nzi;
    double acc = 0.0;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        unsigned i = t % nxi, rest = t / nxi;
        unsigned j = rest % nyi, k = rest / nyi;
        double v = x[g.at(i + 1, j + 1, k + 1)];
        acc = fma(v, v, acc);
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[slot] = sum of partial[0..n) in a fixed order (one block of 256 threads)
__global__ void k_reduce_final(const double *__restrict__ partial, int n, double *out, int slot) {
    __shared__ double sh[8];
    double acc = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) acc += partial[t];
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[slot] = s;
}

// ---------------------------------------------------------------------------
// derivative kernels (FP64)

__device__ __forceinline__ double face_da(double a, double b, int harm) {
    return harm ? 2.0 * b * b / ((a + b) * (a + b)) : 0.5;
}

// Gradients of <w, u> given u and lam = A^{-T} w, on every vertex v:
//   Dbar_v  = -(1/h^2) sum_{j nbr v} dface(D_v, D_j)/dD_v (lam_v - lam_j)(u_v - u_j)
//   mubar_v = -lam_v u_v   (0 on the boundary)
// u and lam are zero on boundary vertices.
__global__ void __launch_bounds__(256) k_grad(Geom g, const double *__restrict__ u,
                                              const double *__restrict__ lam,
                                              const double *__restrict__ D, double ih2, int harm,
                                              double *__restrict__ Dbar, double *__restrict__ mubar) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    long long p = g.at(i, j, k);
    double uv = u[p], lv = lam[p];
    double dv = harm ? D[p] : 0.0;
    double s = 0.0;
    long long off[6] = {-1, 1, -(long long)g.sy, (long long)g.sy, -g.sz, g.sz};
    bool ok[6] = {i > 0, i < g.nx - 1, j > 0, j < g.ny - 1, k > 0, k < g.nz - 1};
#pragma unroll
    for (int n = 0; n < 6; n++) {
        if (!ok[n]) continue;
        long long q = p + off[n];
        double w = harm ? face_da(dv, D[q], 1) : 0.5;
        s = fma(w * (lv - lam[q]), uv - u[q], s);
    }
    if (Dbar) Dbar[p] = -s * ih2;
    if (mubar) mubar[p] = -lv * uv;
}

// f -= (dA) u on interior vertices: the derivative of the operator in the
// direction (dD, dmu) applied to u (either tangent may be NULL).
__global__ void __launch_bounds__(256) k_dA(Geom g, const double *__restrict__ u,
                                            const double *__restrict__ dD,
                                            const double *__restrict__ dmu,
                                            const double *__restrict__ D, double ih2, int harm,
                                            double *__restrict__ f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    long long p = g.at(i, j, k);
    double up = u[p];
    double s = 0.0;
    if (dD) {
        long long off[6] = {-1, 1, -(long long)g.sy, (long long)g.sy, -g.sz, g.sz};
        double dp = D[p], ddp = dD[p];
#pragma unroll
        for (int n = 0; n < 6; n++) {
            long long q = p + off[n];
            double dface = face_da(dp, D[q], harm) * ddp + face_da(D[q], dp, harm) * dD[q];
            s = fma(dface, up - u[q], s);
        }
    }
    double v = s * ih2 + (dmu ? dmu[p] * up : 0.0);
    f[p] -= v;
}

// mixed precision: u64 += s * e32 on interior vertices
__global__ void __launch_bounds__(256) k_update(Geom g, double *__restrict__ u,
                                                const float *__restrict__ e, double s) {
    int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    long long p = g.at(i, j, k);
    u[p] = fma(s, (double)e[p], u[p]);
}

// y = (float)(x * s) on interior vertices
__global__ void __launch_bounds__(256) k_to_f32(Geom g, const double *__restrict__ x, double s,
                                                float *__restrict__ y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k = blockIdx.z + 1;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    long long p = g.at(i, j, k);
    y[p] = (float)(x[p] * s);
}

}  // namespace dmgk
