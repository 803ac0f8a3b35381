// Kernels of the unrolled coefficient gradient: the reverse pass through every
// operation of m FP64 V-cycles (Sec. 2.2), with the coefficients as inputs of
// every level's operator (the extension of the pull-back of Sec. 2.4 to D and
// mu that Sec. 4 names as future work).
//
// Reverse-mode rules used (a_pq = face(D_p, D_q) / h^2 is the coupling stored at
// the lower vertex of each face, diag_p = sum_q a_pq + mu_p):
//   Gauss-Seidel update of p, u_p <- (f_p + sum_q a_pq u_q) / diag_p, with ubar_p
//   the cotangent of the new value and U the state after the half-sweep:
//     t = ubar_p / diag_p;  fbar_p += t;  ubar_q += a_pq t;  abar_pq += t (U_q - U_p);
//     mubar_p -= t U_p;  ubar_p = 0 (the old value is overwritten).
//   Defect r = f - A U with cotangent rbar:  fbar += rbar;  ubar -= A rbar;
//     abar_pq -= (rbar_p - rbar_q)(U_p - U_q);  mubar_p -= rbar_p U_p.
//   Exact coarsest solve u = A^{-1} f with cotangent ubar: fbar = A^{-1} ubar and
//     the same coefficient terms as the defect with rbar := fbar, U := u.
//   Transfers: cotangents move by the transposes, R^T (coarse -> fine) and
//     P^T = 2^3 R (fine -> coarse); coefficient coarsening by its transpose.
// Face cotangents abar are accumulated per face (one writer per face in each
// kernel) and turned into vertex D cotangents at the end, so no kernel needs
// atomics and every sum has a fixed order.
#pragma once

namespace dmgk {

// cotangent of the other colour: for every interior q of colour 1 - color,
// ubar_q += sum over its neighbours p (colour color) of a_pq ubar_p / diag_p
__global__ void __launch_bounds__(256) k_rev_other(Geom g, FaceCoef<double> c, int color, double *__restrict__ ub) {
    int k;
    const int smp = zsplit(g, kInterior, k);
    k += 1;
    const long long o = smp * g.sb;
    ub += o;
    c = c.shifted(o);
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int par = (1 - color + j + k) & 1;
    const int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x) + 2 - par;
    if (j > g.ny - 2 || i > g.nx - 2) return;
    const long long p = g.pos(i, j, k);
    const Nbr n = neighbours(g, i);
    double a[6];
    c.couplings(p, n, a);
    double s = ub[p];
#pragma unroll
    for (int q = 0; q < 6; q++) s = fma(a[q] * __ldg(c.invd + p + n.o[q]), ub[p + n.o[q]], s);
    ub[p] = s;
}

// the updated colour: fbar, mubar and the face cotangents of every vertex p
// of colour `color`, then ubar_p = 0; U is the state after the half-sweep
__global__ void __launch_bounds__(256) k_rev_own(Geom g, FaceCoef<double> c, int color, const double *__restrict__ U,
                                                 double *__restrict__ ub, double *__restrict__ fb,
                                                 double *__restrict__ bx, double *__restrict__ by,
                                                 double *__restrict__ bz, double *__restrict__ mub) {
    int k;
    const int smp = zsplit(g, kInterior, k);
    k += 1;
    const long long o = smp * g.sb;
    U += o; ub += o; fb += o; bx += o; by += o; bz += o; mub += o;
    c = c.shifted(o);
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int par = (color + j + k) & 1;
    const int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x) + 2 - par;
    if (j > g.ny - 2 || i > g.nx - 2) return;
    const long long p = g.pos(i, j, k);
    const Nbr n = neighbours(g, i);
    g.check(p);
#pragma unroll
    for (int q = 0; q < 6; q++) g.check(p + n.o[q]);
    const double t = ub[p] * __ldg(c.invd + p);
    const double up = U[p];
    fb[p] += t;
    mub[p] = fma(-t, up, mub[p]);
    bx[p + n.o[0]] = fma(t, U[p + n.o[0]] - up, bx[p + n.o[0]]);
    bx[p] = fma(t, U[p + n.o[1]] - up, bx[p]);
    by[p + n.o[2]] = fma(t, U[p + n.o[2]] - up, by[p + n.o[2]]);
    by[p] = fma(t, U[p + n.o[3]] - up, by[p]);
    bz[p + n.o[4]] = fma(t, U[p + n.o[4]] - up, bz[p + n.o[4]]);
    bz[p] = fma(t, U[p + n.o[5]] - up, bz[p]);
    ub[p] = 0.0;
}

// defect r = f - A U with cotangent rb: on interior vertices fbar += rb and
// ubar -= A rb (rb zero on the boundary)
__global__ void __launch_bounds__(256) k_rev_defect(Geom g, FaceCoef<double> c, const double *__restrict__ rb,
                                                    double *__restrict__ ub, double *__restrict__ fb) {
    int i = vertex_i();
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k;
    const int smp = zsplit(g, kInterior, k);
    k += 1;
    const long long o = smp * g.sb;
    rb += o; ub += o; fb += o;
    c = c.shifted(o);
    if (i < 1 || i > g.nx - 2 || j > g.ny - 2) return;
    const long long p = g.pos(i, j, k);
    const Nbr n = neighbours(g, i);
    double a[6];
    c.couplings(p, n, a);
    // (A rb)_p = diag_p rb_p - sum_q a_pq rb_q
    double s = -__ldg(c.diag + p) * rb[p];
#pragma unroll
    for (int q = 0; q < 6; q++) s = fma(a[q], rb[p + n.o[q]], s);
    ub[p] += s;
    fb[p] += rb[p];
}

// coefficient cotangents of a defect or of the coarsest solve: for the faces
// (p, p+x), (p, p+y), (p, p+z) stored at p, abar -= (rb_p - rb_q)(U_p - U_q);
// mubar_p -= rb_p U_p on interior p. rb and U are zero on the boundary.
__global__ void __launch_bounds__(256) k_rev_faces(Geom g, const double *__restrict__ rb,
                                                   const double *__restrict__ U, double *__restrict__ bx,
                                                   double *__restrict__ by, double *__restrict__ bz,
                                                   double *__restrict__ mub) {
    int i, j, k, smp;
    if (!vertex_ijk(g, i, j, k, smp)) return;
    const long long o = smp * g.sb;
    rb += o; U += o; bx += o; by += o; bz += o; mub += o;
    const long long p = g.pos(i, j, k);
    const double r = rb[p], u = U[p];
    if (i < g.nx - 1) {
        const long long q = p + g.xp(i);
        bx[p] = fma(-(r - rb[q]), u - U[q], bx[p]);
    }
    if (j < g.ny - 1) {
        const long long q = p + g.sy;
        by[p] = fma(-(r - rb[q]), u - U[q], by[p]);
    }
    if (k < g.nz - 1) {
        const long long q = p + g.sz;
        bz[p] = fma(-(r - rb[q]), u - U[q], bz[p]);
    }
    if (i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1) mub[p] = fma(-r, u, mub[p]);
}

// y += x on interior vertices
__global__ void __launch_bounds__(256) k_add_interior(Geom g, const double *__restrict__ x, double *__restrict__ y) {
    int i = vertex_i();
    int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    int k;
    const int smp = zsplit(g, kInterior, k);
    k += 1;
    if (i < 1 || i > g.nx - 2 || j > g.ny - 2) return;
    const long long p = g.pos(i, j, k) + smp * g.sb;
    y[p] += x[p];
}

__device__ __forceinline__ double face_da64(double a, double b, int harm) {
    return harm ? 2.0 * b * b / ((a + b) * (a + b)) : 0.5;
}

// vertex D cotangents from the face cotangents: a = face(D_v, D_w) / h^2, so
// Dbar_v = sum over the faces of v of abar * dface/dD_v / h^2 (all vertices)
__global__ void __launch_bounds__(256) k_faces_to_vertex(Geom g, const double *__restrict__ D, double ih2, int harm,
                                                         const double *__restrict__ bx, const double *__restrict__ by,
                                                         const double *__restrict__ bz, double *__restrict__ Db) {
    int i, j, k, smp;
    if (!vertex_ijk(g, i, j, k, smp)) return;
    const long long o = smp * g.sb;
    D += o; bx += o; by += o; bz += o; Db += o;
    const long long p = g.pos(i, j, k);
    const double d = D[p];
    double s = 0.0;
    if (i > 0) s = fma(bx[p + g.xm(i)], face_da64(d, D[p + g.xm(i)], harm), s);
    if (i < g.nx - 1) s = fma(bx[p], face_da64(d, D[p + g.xp(i)], harm), s);
    if (j > 0) s = fma(by[p - g.sy], face_da64(d, D[p - g.sy], harm), s);
    if (j < g.ny - 1) s = fma(by[p], face_da64(d, D[p + g.sy], harm), s);
    if (k > 0) s = fma(bz[p - g.sz], face_da64(d, D[p - g.sz], harm), s);
    if (k < g.nz - 1) s = fma(bz[p], face_da64(d, D[p + g.sz], harm), s);
    Db[p] = s * ih2;
}

// 1/4 [1 2 1] weight of the fine offset i - 2I along one axis
__device__ __forceinline__ double fw1(int off) { return off == 0 ? 0.5 : 0.25; }

// Transposes of the two fine-from-coarse maps, gathered at fine vertex (i, j, k):
// sum over the coarse vertices I with |i - 2I| <= 1 (per axis) of
//   interior I:  fw(i-2I) fw(j-2J) fw(k-2K) x_I      (full weighting / restriction)
//   boundary I:  x_I when (i, j, k) = 2I and inject_boundary (coarsening's injection)
// With inject_all, every coarse I contributes by injection only.
__device__ __forceinline__ double gather_T(const Geom &gc, const double *x, int i, int j, int k, bool inject_boundary,
                                           bool inject_all) {
    int Ic[2], Jc[2], Kc[2], ni = 0, nj = 0, nk = 0;
    if (i & 1) { Ic[0] = (i - 1) >> 1; Ic[1] = (i + 1) >> 1; ni = 2; } else { Ic[0] = i >> 1; ni = 1; }
    if (j & 1) { Jc[0] = (j - 1) >> 1; Jc[1] = (j + 1) >> 1; nj = 2; } else { Jc[0] = j >> 1; nj = 1; }
    if (k & 1) { Kc[0] = (k - 1) >> 1; Kc[1] = (k + 1) >> 1; nk = 2; } else { Kc[0] = k >> 1; nk = 1; }
    double s = 0.0;
    for (int c = 0; c < nk; c++)
        for (int b = 0; b < nj; b++)
            for (int a = 0; a < ni; a++) {
                const int I = Ic[a], J = Jc[b], K = Kc[c];
                if (I < 0 || J < 0 || K < 0 || I > gc.nx - 1 || J > gc.ny - 1 || K > gc.nz - 1) continue;
                const bool inner = I > 0 && J > 0 && K > 0 && I < gc.nx - 1 && J < gc.ny - 1 && K < gc.nz - 1;
                const bool at = i == 2 * I && j == 2 * J && k == 2 * K;
                const double v = x[gc.pos(I, J, K)];
                if (inject_all) {
                    if (at) s += v;
                } else if (inner) {
                    s = fma(fw1(i - 2 * I) * fw1(j - 2 * J) * fw1(k - 2 * K), v, s);
                } else if (inject_boundary && at) {
                    s += v;
                }
            }
    return s;
}

// out_f = R^T x_c on fine interior vertices, 0 on the fine boundary
__global__ void __launch_bounds__(256) k_restrict_T(Geom gc, const double *__restrict__ x, Geom gf,
                                                    double *__restrict__ out) {
    int i, j, k, smp;
    if (!vertex_ijk(gf, i, j, k, smp)) return;
    x += smp * gc.sb;
    out += smp * gf.sb;
    const bool inner = i > 0 && j > 0 && k > 0 && i < gf.nx - 1 && j < gf.ny - 1 && k < gf.nz - 1;
    out[gf.pos(i, j, k)] = inner ? gather_T(gc, x, i, j, k, false, false) : 0.0;
}

// Xbar_f += C^T Xbar_c for the coefficient coarsening C (full weighting inside,
// injection on the coarse boundary; inject_all: injection everywhere)
__global__ void __launch_bounds__(256) k_coarsen_T(Geom gc, const double *__restrict__ xc, Geom gf,
                                                   double *__restrict__ xf, int inject_all) {
    int i, j, k, smp;
    if (!vertex_ijk(gf, i, j, k, smp)) return;
    xc += smp * gc.sb;
    xf += smp * gf.sb;
    const long long p = gf.pos(i, j, k);
    xf[p] += gather_T(gc, xc, i, j, k, true, inject_all != 0);
}

// out_c = P^T x_f = 2^3 R x_f on coarse interior vertices (x_f zero on the
// fine boundary), 0 on the coarse boundary
__global__ void __launch_bounds__(256) k_prolong_T(Geom gf, const double *__restrict__ x, Geom gc,
                                                   double *__restrict__ out) {
    int I, J, K, smp;
    if (!vertex_ijk(gc, I, J, K, smp)) return;
    x += smp * gf.sb;
    out += smp * gc.sb;
    const bool inner = I > 0 && J > 0 && K > 0 && I < gc.nx - 1 && J < gc.ny - 1 && K < gc.nz - 1;
    if (!inner) {
        out[gc.pos(I, J, K)] = 0.0;
        return;
    }
    restrict_point(gf, x, gc, out, I, J, K);
    out[gc.pos(I, J, K)] *= 8.0;
}

}  // namespace dmgk
