// Kernels of the two-dimensional solver (the paper's 2D benchmarks, Sec. 3):
// the same method as the 3D kernels on a (ny, nx) vertex grid with the 5-point
// operator, red-black colouring by (i + j) mod 2, full weighting 1/4 [1 2 1]
// per axis (Eq. 7) and prolongation 2^2 R^T (bilinear, Eq. 17).
//
// A 2D level is a Geom with nz == 1: one plane per sample (split rows as in 3D,
// pos(i, j, 0)), sample pitch sb = ny sy, and blockIdx.z = sample. The
// coefficient policies FaceCoef / VertCoef are those of the 3D kernels (the z
// couplings are simply not read).
#pragma once

namespace dmgk {

// couplings of interior vertex p to its -x, +x, -y, +y neighbours
template <class T, bool RO>
__device__ __forceinline__ void couplings2(const FaceCoef<T, RO> &c, long long p, int xm, int sy, T a[4]) {
    a[0] = cld<RO>(c.cx + p + xm);
    a[1] = cld<RO>(c.cx + p);
    a[2] = cld<RO>(c.cy + p - sy);
    a[3] = cld<RO>(c.cy + p);
}
template <class T, bool H, bool RO>
__device__ __forceinline__ void couplings2(const VertCoef<T, H, RO> &c, long long p, int xm, int sy, T a[4]) {
    using V = VertCoef<T, H, RO>;
    const T d = cld<RO>(c.Dh + p);
    a[0] = V::face(d, cld<RO>(c.Dh + p + xm));
    a[1] = V::face(d, cld<RO>(c.Dh + p + xm + 1));
    a[2] = V::face(d, cld<RO>(c.Dh + p - sy));
    a[3] = V::face(d, cld<RO>(c.Dh + p + sy));
}
// note: for FaceCoef the +x coupling is stored at p itself; the -x one at the
// -x neighbour, p + xm. For VertCoef the +x neighbour is p + xm + 1 (split rows).

template <class T, bool RO>
__device__ __forceinline__ T diag2(const FaceCoef<T, RO> &c, long long p, const T *) { return cld<RO>(c.diag + p); }
template <class T, bool H, bool RO>
__device__ __forceinline__ T diag2(const VertCoef<T, H, RO> &c, long long p, const T *a) {
    return (a[0] + a[1]) + ((a[2] + a[3]) + cld<RO>(c.mu + p));
}
template <class T, bool RO>
__device__ __forceinline__ T finish2(const FaceCoef<T, RO> &c, T s, long long p, const T *) {
    return s * cld<RO>(c.invd + p);
}
template <class T, bool H, bool RO>
__device__ __forceinline__ T finish2(const VertCoef<T, H, RO> &c, T s, long long p, const T *a) {
    return __fdividef(s, diag2(c, p, a));
}

// s + sum_q a_q u_q over the four neighbours (FP64: one FMA chain; FP32: two pairs)
template <class T>
__device__ __forceinline__ T coupled_sum2(T s, const T *u, long long p, int xm, int sy, const T *a) {
    if constexpr (sizeof(T) == 8) {
        s = fma(a[0], u[p + xm], s);
        s = fma(a[1], u[p + xm + 1], s);
        s = fma(a[2], u[p - sy], s);
        return fma(a[3], u[p + sy], s);
    } else {
        T s0 = fma(a[0], u[p + xm], s);
        T s1 = a[2] * u[p - sy];
        s0 = fma(a[1], u[p + xm + 1], s0);
        s1 = fma(a[3], u[p + sy], s1);
        return s0 + s1;
    }
}

// Red-black Gauss-Seidel on one colour (Eq. 9): colour = (i + j) mod 2
template <class T, class C>
__global__ void __launch_bounds__(256) k_smooth_half2(Geom g, T *__restrict__ u, const T *__restrict__ f, C c,
                                                      int color, const int *act) {
    pdl_wait();
    const int smp = blockIdx.z;
    if (inactive(act, smp)) return;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int par = (color + j) & 1;
    const int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x) + 2 - par;
    if (j > g.ny - 2 || i > g.nx - 2) return;
    const long long o = smp * g.sb;
    u += o;
    f += o;
    c = c.shifted(o);
    const long long p = g.pos(i, j, 0);
    const int xm = g.xm(i);
    DMG_CHECK(smp < g.nb);
    g.check(p - g.sy);
    g.check(p + g.sy);
    g.check(p + xm);
    g.check(p + xm + 1);
    T a[4];
    couplings2(c, p, xm, g.sy, a);
    u[p] = finish2(c, coupled_sum2(f[p], u, p, xm, g.sy, a), p, a);
}

// The FP32 half-sweep with two vertices per thread (elements m, m+1 of the
// colour's half-row, as the 3D pair kernels): every operand is one 8-byte load
// per pair (own Dh, f, mu; the y neighbours of u and Dh; two of the three x
// neighbours in the other half) plus one 4-byte load. Each vertex repeats the
// arithmetic of couplings2 / coupled_sum2 / diag2 / finish2 in their order, so
// results are bit for bit those of k_smooth_half2<float>.
template <bool HARM>
__global__ void __launch_bounds__(256) k_smooth_half2_pair32(Geom g, float *__restrict__ u,
                                                             const float *__restrict__ f, VertCoef<float, HARM> c,
                                                             int color, const int *act) {
    pdl_wait();
    using V = VertCoef<float, HARM>;
    const int smp = blockIdx.z;
    if (inactive(act, smp)) return;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (j > g.ny - 2) return;
    const int par = (color + j) & 1;   // parity of i for this colour in row j
    const int m = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int i0 = 2 * m + par;
    const bool v0 = i0 >= 1 && i0 <= g.nx - 2, v1 = i0 + 2 <= g.nx - 2;
    if (!v0 && !v1) return;
    const long long o = smp * g.sb;
    u += o;
    f += o;
    const float *Dh = c.Dh + o, *mu = c.mu + o;
    const int row = j * g.sy, sy = g.sy;
    const int p = row + par * g.hx + m, q = row + (1 - par) * g.hx + m;
    const int e = par ? q + 2 : q - 1;   // the third x neighbour
    DMG_CHECK(smp < g.nb);
    g.check(p - sy);
    g.check(p + sy + 1);
    g.check(e);
    g.check(q + 1);
    auto ld = [](const float *x) { return __ldg(reinterpret_cast<const float2 *>(x)); };
    auto lu = [](const float *x) { return *reinterpret_cast<const float2 *>(x); };
    const float2 d = ld(Dh + p), dq = ld(Dh + q), uq = lu(u + q);
    const float de = __ldg(Dh + e), ue = u[e];
    // x neighbours: par 0 (i = 2m): other half m-1, m | m, m+1; par 1 (i = 2m+1): m, m+1 | m+1, m+2
    const float dxm0 = par ? dq.x : de, dxp0 = par ? dq.y : dq.x, dxm1 = par ? dq.y : dq.x, dxp1 = par ? de : dq.y;
    const float uxm0 = par ? uq.x : ue, uxp0 = par ? uq.y : uq.x, uxm1 = par ? uq.y : uq.x, uxp1 = par ? ue : uq.y;
    const float2 dym = ld(Dh + p - sy), dyp = ld(Dh + p + sy), uym = lu(u + p - sy), uyp = lu(u + p + sy);
    const float2 ff = lu(f + p), mm = ld(mu + p);
    auto update = [](float dv, float a0d, float a1d, float a2d, float a3d, float um, float up, float uym_,
                     float uyp_, float fv, float muv) {
        const float a0 = V::face(dv, a0d), a1 = V::face(dv, a1d), a2 = V::face(dv, a2d), a3 = V::face(dv, a3d);
        float s0 = fmaf(a0, um, fv);
        float s1 = a2 * uym_;
        s0 = fmaf(a1, up, s0);
        s1 = fmaf(a3, uyp_, s1);
        const float s = s0 + s1;
        return __fdividef(s, (a0 + a1) + ((a2 + a3) + muv));
    };
    const float r0 = update(d.x, dxm0, dxp0, dym.x, dyp.x, uxm0, uxp0, uym.x, uyp.x, ff.x, mm.x);
    const float r1 = update(d.y, dxm1, dxp1, dym.y, dyp.y, uxm1, uxp1, uym.y, uyp.y, ff.y, mm.y);
    if (v0 && v1) *reinterpret_cast<float2 *>(u + p) = make_float2(r0, r1);
    else if (v0) u[p] = r0;
    else u[p + 1] = r1;
}

// r = f - A u on interior vertices
template <class T, class C>
__global__ void __launch_bounds__(256) k_residual2(Geom g, const T *__restrict__ u, const T *__restrict__ f, C c,
                                                   T *__restrict__ r, const int *act) {
    const int smp = blockIdx.z;
    if (inactive(act, smp)) return;
    const int i = vertex_i();
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i < 1 || i > g.nx - 2 || j > g.ny - 2) return;
    const long long o = smp * g.sb;
    u += o;
    f += o;
    r += o;
    c = c.shifted(o);
    const long long p = g.pos(i, j, 0);
    const int xm = g.xm(i);
    T a[4];
    couplings2(c, p, xm, g.sy, a);
    r[p] = coupled_sum2(fma(-diag2(c, p, a), u[p], f[p]), u, p, xm, g.sy, a);
}

// f_c = R r (9-point full weighting) and u_c = 0 on coarse interior vertices
template <class T>
__global__ void __launch_bounds__(256) k_restrict2(Geom gf, const T *__restrict__ r, Geom gc, T *__restrict__ fc,
                                                   T *__restrict__ uc, const int *act) {
    const int smp = blockIdx.z;
    if (inactive(act, smp)) return;
    const int I = vertex_i();
    const int J = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (I < 1 || I > gc.nx - 2 || J > gc.ny - 2) return;
    r += smp * gf.sb;
    const long long pc = gc.pos(I, J, 0) + smp * gc.sb;
    const long long p = gf.pos(2 * I, 2 * J, 0);
    const int om = gf.xm(2 * I), op = gf.xp(2 * I);
    T s = T(0);
#pragma unroll
    for (int b = -1; b <= 1; b++) {
        const long long q = p + b * gf.sy;
        const T row = r[q + om] + T(2) * r[q] + r[q + op];
        s += (b == 0 ? T(2) : T(1)) * row;
    }
    gf.check(p - gf.sy + om);
    gf.check(p + gf.sy + op);
    gc.check(gc.pos(I, J, 0));
    fc[pc] = s * T(1.0 / 16.0);
    uc[pc] = T(0);
}

// u += P e on the fine vertices of one coarse cell (I..I+1, J..J+1), bilinear
template <class T>
__global__ void __launch_bounds__(256) k_prolong_add2(Geom gc, const T *__restrict__ e, Geom gf, T *__restrict__ u,
                                                      const int *act) {
    pdl_wait();
    const int smp = blockIdx.z;
    if (inactive(act, smp)) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I > gc.nx - 2 || J > gc.ny - 2) return;
    e += smp * gc.sb;
    u += smp * gf.sb;
    T c[2][2];
#pragma unroll
    for (int y = 0; y < 2; y++)
#pragma unroll
        for (int x = 0; x < 2; x++) c[y][x] = e[gc.pos(I + x, J + y, 0)];
#pragma unroll
    for (int by = 0; by < 2; by++) {
        const int j = 2 * J + by;
        if (j < 1 || j > gf.ny - 2) continue;
        T row[2];
#pragma unroll
        for (int x = 0; x < 2; x++) row[x] = by ? T(0.5) * (c[0][x] + c[1][x]) : c[0][x];
        if (2 * I >= 1) u[gf.pos(2 * I, j, 0)] += row[0];
        if (2 * I + 1 <= gf.nx - 2) u[gf.pos(2 * I + 1, j, 0)] += T(0.5) * (row[0] + row[1]);
    }
}

// After a half-sweep the defect vanishes on the colour it updated (as in 3D):
// r = f - A u is formed on the other colour only (colour = (i + j) mod 2, one
// vertex per thread as k_smooth_half2), and the restriction below reads only
// that colour.
template <class T, class C>
__global__ void __launch_bounds__(256) k_residual_colour2(Geom g, const T *__restrict__ u, const T *__restrict__ f,
                                                          C c, T *__restrict__ r, int color, const int *act) {
    pdl_wait();
    const int smp = blockIdx.z;
    if (inactive(act, smp)) return;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int par = (color + j) & 1;
    const int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x) + 2 - par;
    if (j > g.ny - 2 || i > g.nx - 2) return;
    const long long o = smp * g.sb;
    u += o;
    f += o;
    r += o;
    c = c.shifted(o);
    const long long p = g.pos(i, j, 0);
    const int xm = g.xm(i);
    DMG_CHECK(smp < g.nb);
    g.check(p - g.sy);
    g.check(p + g.sy);
    g.check(p + xm);
    g.check(p + xm + 1);
    T a[4];
    couplings2(c, p, xm, g.sy, a);
    r[p] = coupled_sum2(fma(-diag2(c, p, a), u[p], f[p]), u, p, xm, g.sy, a);
}

// 9-point full weighting of a defect that lives on one colour: fine vertex
// (2I+a, 2J+b) has colour (a+b) mod 2, so in row b either the centre (a = 0)
// or the two sides (a = -1, +1) carry it (PAR: the colour of the defect).
template <class T, int PAR>
__global__ void __launch_bounds__(256) k_restrict_colour2(Geom gf, const T *__restrict__ r, Geom gc,
                                                          T *__restrict__ fc, T *__restrict__ uc, const int *act) {
    pdl_wait();
    const int smp = blockIdx.z;
    if (inactive(act, smp)) return;
    const int I = vertex_i();
    const int J = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (I < 1 || I > gc.nx - 2 || J > gc.ny - 2) return;
    r += smp * gf.sb;
    const long long pc = gc.pos(I, J, 0) + smp * gc.sb;
    const long long p = gf.pos(2 * I, 2 * J, 0);
    const int om = gf.xm(2 * I), op = gf.xp(2 * I);
    gf.check(p - gf.sy + om);
    gf.check(p + gf.sy + op);
    gc.check(gc.pos(I, J, 0));
    T s = T(0);
#pragma unroll
    for (int b = -1; b <= 1; b++) {
        const long long q = p + b * gf.sy;
        const T row = ((b & 1) == PAR) ? T(2) * r[q] : r[q + om] + r[q + op];
        s += (b == 0 ? T(2) : T(1)) * row;
    }
    fc[pc] = s * T(1.0 / 16.0);
    uc[pc] = T(0);
}

// u += P e on the vertices of one colour only (the values the half-sweep of the
// other colour, which must follow, reads); each vertex gets the interpolation
// of k_prolong_add2 in its order, so the level ends bit for bit where the full
// correction and two half-sweeps end.
template <class T>
__global__ void __launch_bounds__(256) k_prolong_colour2(Geom gc, const T *__restrict__ e, Geom gf,
                                                         T *__restrict__ u, int color, const int *act) {
    pdl_wait();
    const int smp = blockIdx.z;
    if (inactive(act, smp)) return;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int par = (color + j) & 1;
    const int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x) + 2 - par;
    if (j > gf.ny - 2 || i > gf.nx - 2) return;
    e += smp * gc.sb;
    u += smp * gf.sb;
    const int I = i >> 1, J = j >> 1, x = i & 1, y = j & 1;
    gc.check(gc.pos(I + x, J + y, 0));
    // the coarse values of the cell (I, J) that k_prolong_add2 reads for this vertex
    const T c00 = e[gc.pos(I, J, 0)];
    T row0 = c00, row1 = T(0);
    if (y) row0 = T(0.5) * (c00 + e[gc.pos(I, J + 1, 0)]);
    if (x) {
        const T c01 = e[gc.pos(I + 1, J, 0)];
        row1 = y ? T(0.5) * (c01 + e[gc.pos(I + 1, J + 1, 0)]) : c01;
    }
    u[gf.pos(i, j, 0)] += x ? T(0.5) * (row0 + row1) : row0;
}

// exact coarsest solve u = Ainv f on the (nx-2)(ny-2) interior unknowns (x fastest), one block per sample
template <class T>
__global__ void k_coarse_solve2(Geom g, const T *__restrict__ Ainv, int n, const T *__restrict__ f,
                                T *__restrict__ u, const int *act) {
    extern __shared__ unsigned char smem_raw[];
    T *fs = reinterpret_cast<T *>(smem_raw);
    const int smp = blockIdx.x;
    if (inactive(act, smp)) return;
    Ainv += (long long)smp * n * n;
    f += smp * g.sb;
    u += smp * g.sb;
    const int nxi = g.nx - 2;
    for (int q = threadIdx.x; q < n; q += blockDim.x) fs[q] = f[g.pos(q % nxi + 1, q / nxi + 1, 0)];
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        T s = T(0);
        for (int q = 0; q < n; q++) s = fma(Ainv[(long long)r * n + q], fs[q], s);
        u[g.pos(r % nxi + 1, r / nxi + 1, 0)] = s;
    }
}

// dense coarsest matrix [A | I] (row stride 2n) from the FP64 faces; blockIdx.y = sample
__global__ void k_coarse_assemble2(Geom g, FaceCoef<double> c, int n, double *M) {
    const int nxi = g.nx - 2;
    c = c.shifted(blockIdx.y * g.sb);
    M += (long long)blockIdx.y * 2 * n * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * 2 * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(t / (2 * n)), col = (int)(t % (2 * n));
        double v = 0.0;
        if (col >= n) {
            v = (col - n == r) ? 1.0 : 0.0;
        } else {
            const int ri = r % nxi + 1, rj = r / nxi + 1, ci = col % nxi + 1, cj = col / nxi + 1;
            const long long p = g.pos(ri, rj, 0);
            const int di = ci - ri, dj = cj - rj;
            if (di == 0 && dj == 0) v = c.diag[p];
            else if (dj == 0 && di == -1) v = -c.cx[p + g.xm(ri)];
            else if (dj == 0 && di == 1) v = -c.cx[p];
            else if (di == 0 && dj == -1) v = -c.cy[p - g.sy];
            else if (di == 0 && dj == 1) v = -c.cy[p];
        }
        M[t] = v;
    }
}

// all vertices of every sample of a 2D level: blockIdx.z = sample
__device__ __forceinline__ bool vertex_ij2(const Geom &g, int &i, int &j) {
    i = vertex_i();
    j = blockIdx.y * blockDim.y + threadIdx.y;
    return i < g.nx && j < g.ny;
}

// coefficient coarsening: full weighting on coarse interior vertices, injection on the coarse boundary
__global__ void k_coarsen2(Geom gf, const double *__restrict__ X, Geom gc, double *__restrict__ Xc, int inject) {
    int I, J;
    if (!vertex_ij2(gc, I, J)) return;
    X += blockIdx.z * gf.sb;
    Xc += blockIdx.z * gc.sb;
    const bool inner = I > 0 && J > 0 && I < gc.nx - 1 && J < gc.ny - 1;
    const long long p = gf.pos(2 * I, 2 * J, 0);
    double s;
    if (inject || !inner) {
        s = X[p];
    } else {
        const int om = gf.xm(2 * I), op = gf.xp(2 * I);
        s = 0.0;
        for (int b = -1; b <= 1; b++) {
            const long long q = p + b * gf.sy;
            const double row = 0.25 * X[q + om] + 0.5 * X[q] + 0.25 * X[q + op];
            s += (b == 0 ? 0.5 : 0.25) * row;
        }
    }
    Xc[gc.pos(I, J, 0)] = s;
}

// FP64 faces (cx at the lower vertex of each x face, cy of each y face, / h^2), diag and 1/diag
__global__ void k_build_faces2(Geom g, const double *__restrict__ D, const double *__restrict__ mu, double ih2,
                               int harm, double *cx, double *cy, double *diag, double *invd) {
    int i, j;
    if (!vertex_ij2(g, i, j)) return;
    const long long o = blockIdx.z * g.sb, p = g.pos(i, j, 0);
    D += o; mu += o; cx += o; cy += o; diag += o; invd += o;
    const double d = D[p];
    cx[p] = i < g.nx - 1 ? face_mean(d, D[p + g.xp(i)], harm) * ih2 : 0.0;
    cy[p] = j < g.ny - 1 ? face_mean(d, D[p + g.sy], harm) * ih2 : 0.0;
    if (i > 0 && j > 0 && i < g.nx - 1 && j < g.ny - 1) {
        const double s = face_mean(d, D[p + g.xm(i)], harm) + face_mean(d, D[p + g.xp(i)], harm) +
                         face_mean(d, D[p - g.sy], harm) + face_mean(d, D[p + g.sy], harm);
        const double dg = s * ih2 + mu[p];
        diag[p] = dg;
        invd[p] = 1.0 / dg;
    } else {
        diag[p] = 0.0;
        invd[p] = 0.0;
    }
}

// partial[s][b] = sum over block b's interior vertices of sample s of (f - A u)^2;
// optional r32 = r * 2^-e_prev (mixed precision); blockIdx.y = sample
template <class T, class C>
__global__ void __launch_bounds__(256) k_resid_norm2(Geom g, const T *__restrict__ u, const T *__restrict__ f, C c,
                                                     float *__restrict__ r32, const MixScalars *ms, double *partial,
                                                     const int *act) {
    __shared__ double sh[8];
    const int smp = blockIdx.y;
    if (inactive(act, smp)) return;
    const long long o = smp * g.sb;
    u += o;
    f += o;
    c = c.shifted(o);
    if (r32) r32 += o;
    partial += smp * gridDim.x;
    const int nxi = g.nx - 2;
    const unsigned total = (unsigned)nxi * (g.ny - 2);
    const int shift = r32 ? -ms[smp].e_prev : 0;
    double acc = 0.0;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned jj = t / nxi;
        const int i = (int)(t - jj * nxi) + 1, j = (int)jj + 1;
        const long long p = g.pos(i, j, 0);
        const int xm = g.xm(i);
        T a[4];
        couplings2(c, p, xm, g.sy, a);
        const T r = coupled_sum2(fma(-diag2(c, p, a), u[p], f[p]), u, p, xm, g.sy, a);
        if (r32) r32[p] = f64_to_f32_shift((double)r, shift);
        acc = fma((double)r, (double)r, acc);
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// partial[s][b] = sum over block b's interior vertices of sample s of x^2
__global__ void __launch_bounds__(256) k_norm2_2d(Geom g, const double *__restrict__ x, double *partial) {
    __shared__ double sh[8];
    x += blockIdx.y * g.sb;
    partial += blockIdx.y * gridDim.x;
    const int nxi = g.nx - 2;
    const unsigned total = (unsigned)nxi * (g.ny - 2);
    double acc = 0.0;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned jj = t / nxi;
        const double v = x[g.pos((int)(t - jj * nxi) + 1, (int)jj + 1, 0)];
        acc = fma(v, v, acc);
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// gradients of <w, u> from u and lam = A^{-1} w on every vertex (u, lam zero on the boundary):
//   Dbar_v = -(1/h^2) sum_{j nbr v} dface/dD_v (lam_v - lam_j)(u_v - u_j),  mubar_v = -lam_v u_v
__global__ void __launch_bounds__(256) k_grad2(Geom g, const double *__restrict__ u, const double *__restrict__ lam,
                                               const double *__restrict__ D, double ih2, int harm,
                                               double *__restrict__ Dbar, double *__restrict__ mubar) {
    int i, j;
    if (!vertex_ij2(g, i, j)) return;
    const long long o = blockIdx.z * g.sb, p = g.pos(i, j, 0);
    u += o; lam += o; D += o;
    const double uv = u[p], lv = lam[p], dv = D[p];
    double s = 0.0;
    const long long nb[4] = {i > 0 ? p + g.xm(i) : -1, i < g.nx - 1 ? p + g.xp(i) : -1, j > 0 ? p - g.sy : -1,
                             j < g.ny - 1 ? p + g.sy : -1};
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (nb[q] < 0) continue;
        const double w = harm ? face_da(dv, D[nb[q]], 1) : 0.5;
        s = fma(w * (lv - lam[nb[q]]), uv - u[nb[q]], s);
    }
    if (Dbar) Dbar[o + p] = -s * ih2;
    if (mubar) mubar[o + p] = -lv * uv;
}

// k_grad2 for the arithmetic face mean with each face's operands formed once:
// k_grad2 multiplies (1/2)(lam_v - lam_n) by (u_v - u_n) on every face, and the
// other vertex of the face forms their exact negations (IEEE subtraction and
// scaling are antisymmetric; fma(-a, -b, s) = fma(a, b, s)). A block of
// kGrad2TX x kGrad2TY vertices forms its +x and +y faces' operands once and
// shares them through shared memory; only the -x and -y faces across the
// tile's lower sides are formed again. Bitwise k_grad2's results with about 12
// FP64 operations per vertex against 18. dnat, mnat: that output is written in
// the caller's natural layout (x fastest, samples consecutive).
constexpr int kGrad2TX = 32, kGrad2TY = 8;

__global__ void __launch_bounds__(kGrad2TX * kGrad2TY) k_grad2_am(Geom g, const double *__restrict__ u,
                                                                  const double *__restrict__ lam, double ih2,
                                                                  double *__restrict__ Dbar, bool dnat,
                                                                  double *__restrict__ mubar, bool mnat) {
    __shared__ double su[kGrad2TY][kGrad2TX], sl[kGrad2TY][kGrad2TX];
    __shared__ double hl2[2][kGrad2TY][kGrad2TX], du2[2][kGrad2TY][kGrad2TX];
    const int tx = threadIdx.x, ty = threadIdx.y, smp = blockIdx.z;
    const int i = blockIdx.x * kGrad2TX + tx, j = blockIdx.y * kGrad2TY + ty;
    const bool in = i < g.nx && j < g.ny;
    const long long o = smp * g.sb;
    u += o;
    lam += o;
    const long long p = in ? g.pos(i, j, 0) : 0;
    double uv = 0.0, lv = 0.0;
    if (in) {
        g.check(p);
        uv = u[p];
        lv = lam[p];
    }
    su[ty][tx] = uv;
    sl[ty][tx] = lv;
    __syncthreads();
    const bool up[2] = {in && i < g.nx - 1, in && j < g.ny - 1};
    const bool last[2] = {tx == kGrad2TX - 1, ty == kGrad2TY - 1};
    const long long po[2] = {g.xp(i), g.sy};
    double hlp[2], dup[2];
#pragma unroll
    for (int a = 0; a < 2; a++) {
        double un = 0.0, ln = 0.0;
        if (up[a]) {
            if (last[a]) {
                g.check(p + po[a]);
                un = u[p + po[a]];
                ln = lam[p + po[a]];
            } else {
                un = a == 0 ? su[ty][tx + 1] : su[ty + 1][tx];
                ln = a == 0 ? sl[ty][tx + 1] : sl[ty + 1][tx];
            }
        }
        hlp[a] = 0.5 * (lv - ln);
        dup[a] = uv - un;
        hl2[a][ty][tx] = hlp[a];
        du2[a][ty][tx] = dup[a];
    }
    __syncthreads();
    if (!in) return;
    const bool dn[2] = {i > 0, j > 0};
    const bool first[2] = {tx == 0, ty == 0};
    const long long mo[2] = {g.xm(i), -(long long)g.sy};
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 2; a++) {
        if (dn[a]) {
            double hm, dm;
            if (first[a]) {
                g.check(p + mo[a]);
                hm = 0.5 * (lv - lam[p + mo[a]]);
                dm = uv - u[p + mo[a]];
            } else {
                hm = a == 0 ? hl2[0][ty][tx - 1] : hl2[1][ty - 1][tx];
                dm = a == 0 ? du2[0][ty][tx - 1] : du2[1][ty - 1][tx];
            }
            s = fma(hm, dm, s);
        }
        if (up[a]) s = fma(hlp[a], dup[a], s);
    }
    const long long nat = ((long long)smp * g.ny + j) * g.nx + i;
    DMG_CHECK(nat < (long long)g.nb * g.ny * g.nx);
    if (Dbar) Dbar[dnat ? nat : o + p] = -s * ih2;
    if (mubar) mubar[mnat ? nat : o + p] = -lv * uv;
}

// f -= (dA) u on interior vertices for a coefficient direction (dD, dmu)
__global__ void __launch_bounds__(256) k_dA2(Geom g, const double *__restrict__ u, const double *__restrict__ dD,
                                             const double *__restrict__ dmu, const double *__restrict__ D, double ih2,
                                             int harm, double *__restrict__ f) {
    const int i = vertex_i();
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i < 1 || i > g.nx - 2 || j > g.ny - 2) return;
    const long long o = blockIdx.z * g.sb, p = g.pos(i, j, 0);
    u += o; D += o; f += o;
    if (dD) dD += o;
    if (dmu) dmu += o;
    const double up = u[p];
    double s = 0.0;
    if (dD) {
        const double dp = D[p], ddp = dD[p];
        const long long nb[4] = {p + g.xm(i), p + g.xp(i), p - g.sy, p + g.sy};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const long long r = nb[q];
            const double dface = face_da(dp, D[r], harm) * ddp + face_da(D[r], dp, harm) * dD[r];
            s = fma(dface, up - u[r], s);
        }
    }
    f[p] -= s * ih2 + (dmu ? dmu[p] * up : 0.0);
}

}  // namespace dmgk
