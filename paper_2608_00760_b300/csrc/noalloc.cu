// dmg_residual_static: the FP64 residual norm ||q - A u||_2 (and ||q||_2)
// computed straight from the caller's device arrays, with no context and no
// device allocation of any kind.
//
// It is meant for callers that may not allocate device memory: a host
// framework that owns the whole device pool through its own allocator and
// forbids cudaMalloc after start-up, or a latency-critical loop where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// Such callers cannot run dmg_setup either, so this entry point needs nothing
// but the arrays they already hold.
//
// The scratch of its two-stage deterministic reduction (one partial sum per
// interior grid row, then one fixed-order final sum) lives in the file-scope
// array below, which every GPU that loads the library holds until exit.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/dmg.h"

// Interior rows ((ny-2)*(nz-2)) one call may cover: 2^18, so 513^3 fits.
#define DMG_STATIC_MAX_ROWS (1 << 18)
#define DMG_STATIC_MAX_DEVICES 64

// [0, MAX): per-row sums of r^2; [MAX, 2 MAX): per-row sums of q^2;
// [2 MAX, 2 MAX + 2): the two norms. 4 MB in total.
static __device__ __align__(256) double dmg_static_scratch[2 * DMG_STATIC_MAX_ROWS + 2];

void dmg_detail_set_noctx_error(const char *msg);  // defined in dmg.cu

namespace {

// contiguous caller layout: element (i, j, k) at k*sz + j*sy + i
struct Grid {
    int nx, ny, nz, sy;
    long long sz;
    __device__ __forceinline__ long long at(int i, int j, int k) const {
        return (long long)k * sz + (long long)j * sy + i;
    }
};

std::mutex g_static_mu;
double *g_static_ptr[DMG_STATIC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once per
// device (the first call on that device) and kept for the life of the process.
// In host code the array's name is only a host-side handle; kernels must be
// given this address. A cudaDeviceReset() unloads the module that holds the
// array, so the kept address would be stale afterwards: this entry point does
// not support being used across a device reset.
dmg_status static_scratch(int dev, double **out) {
    if (dev < 0 || dev >= DMG_STATIC_MAX_DEVICES) {
        dmg_detail_set_noctx_error("dmg_residual_static: device ordinal out of range");
        return DMG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, dmg_static_scratch);
        if (e != cudaSuccess || !p) {
            char m[256];
            snprintf(m, sizeof(m), "dmg_residual_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            dmg_detail_set_noctx_error(m);
            return DMG_ECUDA;
        }
        g_static_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_static_ptr[dev];
    return DMG_OK;
}

__device__ __forceinline__ double face_static(double a, double b, int harm) {
    return harm ? 2.0 * a * b / (a + b) : a + b;
}

// Block sums of two values; valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &b) {
    __shared__ double sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) { x += sa[q]; y += sb[q]; }
        a = x;
        b = y;
    }
}

// One block per interior row (j, k): partial sums of r^2 and q^2 over the row,
// with r = q - A u formed from the vertex coefficients (faces on the fly, u
// taken as zero on boundary vertices).
__global__ void __launch_bounds__(128) k_static_rows(Grid g, const double *__restrict__ D,
                                                     const double *__restrict__ mu,
                                                     const double *__restrict__ q,
                                                     const double *__restrict__ u, double s, int harm,
                                                     double *scratch) {
    int nyi = g.ny - 2;
    int row = blockIdx.x;
    int j = row % nyi + 1, k = row / nyi + 1;
    double ar = 0.0, aq = 0.0;
    for (int i = 1 + threadIdx.x; i <= g.nx - 2; i += blockDim.x) {
        long long p = g.at(i, j, k);
        double dp = D[p], up = u[p];
        long long off[6] = {-1, 1, -(long long)g.sy, (long long)g.sy, -g.sz, g.sz};
        bool in[6] = {i > 1, i < g.nx - 2, j > 1, j < g.ny - 2, k > 1, k < g.nz - 2};
        double au = mu[p] * up;
#pragma unroll
        for (int n = 0; n < 6; n++) {
            double un = in[n] ? u[p + off[n]] : 0.0;
            au = fma(face_static(dp, D[p + off[n]], harm) * s, up - un, au);
        }
        double r = q[p] - au;
        ar = fma(r, r, ar);
        aq = fma(q[p], q[p], aq);
    }
    block_sum2(ar, aq);
    if (threadIdx.x == 0) {
        scratch[row] = ar;
        scratch[DMG_STATIC_MAX_ROWS + row] = aq;
    }
}

// Fixed-order final sums of the rows' partials; writes the two norms.
__global__ void __launch_bounds__(256) k_static_final(double *scratch, int rows) {
    double ar = 0.0, aq = 0.0;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        ar += scratch[t];
        aq += scratch[DMG_STATIC_MAX_ROWS + t];
    }
    block_sum2(ar, aq);
    if (threadIdx.x == 0) {
        scratch[2 * DMG_STATIC_MAX_ROWS] = sqrt(ar);
        scratch[2 * DMG_STATIC_MAX_ROWS + 1] = sqrt(aq);
    }
}

// The runtime keeps one "last error" per host thread. This file never reads it
// with cudaGetLastError(), which would also clear an error that the caller's
// earlier, unrelated work left pending; every runtime call here is checked by
// its own return value instead.
bool on_current_device(const void *ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) return false;
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" dmg_status dmg_residual_static(const dmg_params *p, const double *D, const double *mu,
                                          const double *q, const double *u, double *out, void *stream) {
    char m[256];
    if (!p || !D || !mu || !q || !u || !out) {
        dmg_detail_set_noctx_error("dmg_residual_static: NULL argument");
        return DMG_EINVAL;
    }
    if (p->nx < 3 || p->ny < 3 || p->nz < 3 || (long long)p->nx * p->ny * p->nz > (1LL << 31) - 1 ||
        !(p->h > 0.0) || !std::isfinite(p->h) ||
        (p->face_mean != DMG_FACE_ARITHMETIC && p->face_mean != DMG_FACE_HARMONIC)) {
        dmg_detail_set_noctx_error("dmg_residual_static: invalid nx, ny, nz, h or face_mean");
        return DMG_EINVAL;
    }
    long long rows = (long long)(p->ny - 2) * (p->nz - 2);
    if (rows > DMG_STATIC_MAX_ROWS) {
        snprintf(m, sizeof(m),
                 "dmg_residual_static: grid %dx%dx%d has %lld interior rows; the fixed scratch holds at most %d",
                 p->nx, p->ny, p->nz, rows, DMG_STATIC_MAX_ROWS);
        dmg_detail_set_noctx_error(m);
        return DMG_EINVAL;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        dmg_detail_set_noctx_error("dmg_residual_static: no CUDA device");
        return DMG_ECUDA;
    }
    if (!on_current_device(D, dev) || !on_current_device(mu, dev) || !on_current_device(q, dev) ||
        !on_current_device(u, dev)) {
        dmg_detail_set_noctx_error("dmg_residual_static: D, mu, q and u must be device memory of the current device");
        return DMG_EINVAL;
    }
    double *scratch = nullptr;
    dmg_status st = static_scratch(dev, &scratch);
    if (st != DMG_OK) return st;
    Grid g;
    g.nx = p->nx; g.ny = p->ny; g.nz = p->nz;
    g.sy = p->nx;
    g.sz = (long long)p->nx * p->ny;
    int harm = p->face_mean == DMG_FACE_HARMONIC;
    double s = harm ? 1.0 / (p->h * p->h) : 0.5 / (p->h * p->h);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    // every slot the final kernel reads is written by k_static_rows first, so
    // nothing has to be cleared between calls. Each launch is checked by the
    // status cudaLaunchKernel returns for it.
    const double *cD = D, *cmu = mu, *cq = q, *cu = u;
    void *rows_args[] = {&g, &cD, &cmu, &cq, &cu, &s, &harm, &scratch};
    cudaError_t e = cudaLaunchKernel((const void *)k_static_rows, dim3((unsigned)rows), dim3(128), rows_args, 0, cs);
    int nrows = (int)rows;
    void *final_args[] = {&scratch, &nrows};
    if (e == cudaSuccess) e = cudaLaunchKernel((const void *)k_static_final, dim3(1), dim3(256), final_args, 0, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, scratch + 2 * DMG_STATIC_MAX_ROWS, 2 * sizeof(double), cudaMemcpyDefault, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        snprintf(m, sizeof(m), "dmg_residual_static: %s", cudaGetErrorString(e));
        dmg_detail_set_noctx_error(m);
        return DMG_ECUDA;
    }
    return DMG_OK;
}
