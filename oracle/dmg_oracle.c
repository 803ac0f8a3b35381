/*
 * FP64 CPU oracle for the differentiable multigrid solver (DMGS) of
 * arXiv 2608.00760. TEST INFRASTRUCTURE ONLY: nothing in the product package
 * links, imports or calls this file. It shares no code, header or constant
 * with the CUDA path; the two meet only through the seeded inputs.
 *
 * Everything here is plain, slow, obviously-correct loops in double
 * precision, compiled with -ffp-contract=off. Arrays are dense C-order
 * [nz][ny][nx] over ALL vertices including the two Dirichlet boundary planes
 * of every axis; boundary values of u, f, lambda are zero by definition.
 *
 * What it computes, and where the paper states it:
 *   - the operator of Eq. 1,  (-div(D grad) + mu) u = q, discretised with
 *     second-order central differences (Sec. 2, text after Eq. 1), 7-point,
 *     face coefficient = mean of the two vertex values (arithmetic by default,
 *     harmonic as an option: the paper defers the exact form to the PICARD
 *     reference, so the mean is a reading);
 *   - the grid hierarchy h_k = 2 h_{k-1} with rediscretised L^k per level
 *     (Sec. 2.2, Eq. 6 and the text after it);
 *   - Red-Black Gauss-Seidel, red = even (i+j+k) first (Sec. 2.2, Sec. 2.3.1
 *     Eq. 9) and its per-point adjoint (Eqs. 10-11);
 *   - the defect e = q - L rho and its restriction (Sec. 2.3.2, Eqs. 12-14;
 *     adjoint Eqs. 15-16);
 *   - full-weighting restriction 1/4[1 2 1] per axis (Eq. 7) and the
 *     prolongation I = 2^n R^T (Sec. 2.3.3, Eq. 17);
 *   - the V-cycle composition S = g_l o ... o g_1 repeated (Eq. 5) and its
 *     adjoint as the reversed composition of per-operation adjoints (Sec. 2.4,
 *     Eq. 18), implemented TWICE: literally (orc_adjoint_literal, each forward
 *     operation transposed, run in reverse order) and as the transposed
 *     V-cycle iteration (orc_adjoint), which must agree to rounding;
 *   - the coefficient gradients Dbar, mubar of the converged solution (an
 *     extension: the paper lists differentiation w.r.t. D and the absorption
 *     as future work in Sec. 4) and the tangent operator dA u for the JVP.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   coefficient coarsening = full weighting of vertex D, mu on coarse interior
 *   vertices and injection on the coarse boundary (or pure injection);
 *   coarsest level solved exactly by dense Cholesky of L^{coarsest};
 *   stopping rule ||q - A u||_2 / ||q||_2 over interior vertices.
 *
 * Parity status: every function here is pinned by a CPU test (closed-form
 * eigenmodes, the PDE itself to O(h^2), a library sparse direct solve,
 * brute-force transposes, finite differences, trilinear reproduction), and a
 * mutation test compiles copies of this file with single planted mistakes and
 * requires each copy to fail one of those pins.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXLEV 16

static size_t at(int nx, int ny, int i, int j, int k) {
    return ((size_t)k * (size_t)ny + (size_t)j) * (size_t)nx + (size_t)i;
}

static int is_interior(int nx, int ny, int nz, int i, int j, int k) {
    return i > 0 && j > 0 && k > 0 && i < nx - 1 && j < ny - 1 && k < nz - 1;
}

/* Face coefficient between two vertices: the mean of the vertex values. */
double orc_face(double a, double b, int harmonic) {
    if (harmonic) return 2.0 * a * b / (a + b);
    return 0.5 * (a + b);
}

/* d face / d a */
static double orc_face_da(double a, double b, int harmonic) {
    if (harmonic) return 2.0 * b * b / ((a + b) * (a + b));
    return 0.5;
}

static const int NB[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                             {0, 1, 0},  {0, 0, -1}, {0, 0, 1}};

/* value of a field at a vertex, zero outside the interior (Dirichlet) */
static double val0(int nx, int ny, int nz, const double *u, int i, int j, int k) {
    if (!is_interior(nx, ny, nz, i, j, k)) return 0.0;
    return u[at(nx, ny, i, j, k)];
}

/*
 * out = A u on interior vertices, 0 on the boundary (Eq. 1 discretised):
 *   (A u)_p = (1/h^2) sum_{j in nbr(p)} Dface(p,j) (u_p - u_j) + mu_p u_p
 */
void orc_apply(int nx, int ny, int nz, double h, int harmonic, const double *D,
               const double *mu, const double *u, double *out) {
    double ih2 = 1.0 / (h * h);
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t p = at(nx, ny, i, j, k);
                if (!is_interior(nx, ny, nz, i, j, k)) { out[p] = 0.0; continue; }
                double up = u[p];
                double s = 0.0;
                for (int n = 0; n < 6; n++) {
                    int a = i + NB[n][0], b = j + NB[n][1], c = k + NB[n][2];
                    double fc = orc_face(D[p], D[at(nx, ny, a, b, c)], harmonic);
                    s += fc * (up - val0(nx, ny, nz, u, a, b, c));
                }
                out[p] = s * ih2 + mu[p] * up;
            }
}

/* r = f - A u (defect, Eqs. 13-14), interior only, boundary 0 */
void orc_residual(int nx, int ny, int nz, double h, int harmonic, const double *D,
                  const double *mu, const double *f, const double *u, double *r) {
    orc_apply(nx, ny, nz, h, harmonic, D, mu, u, r);
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t p = at(nx, ny, i, j, k);
                r[p] = is_interior(nx, ny, nz, i, j, k) ? f[p] - r[p] : 0.0;
            }
}

/* diagonal entry of A at p */
static double diag_at(int nx, int ny, double h, int harmonic, const double *D,
                      const double *mu, int i, int j, int k) {
    size_t p = at(nx, ny, i, j, k);
    double s = 0.0;
    for (int n = 0; n < 6; n++)
        s += orc_face(D[p], D[at(nx, ny, i + NB[n][0], j + NB[n][1], k + NB[n][2])],
                      harmonic);
    return s / (h * h) + mu[p];
}

/*
 * One Gauss-Seidel half-sweep over the vertices of one colour (Eq. 9),
 * colour = (i+j+k) mod 2, red = 0. Points of one colour are not neighbours
 * in the 7-point stencil, so the order inside the loop does not matter.
 */
void orc_gs_half(int nx, int ny, int nz, double h, int harmonic, const double *D,
                 const double *mu, const double *f, double *u, int color) {
    double ih2 = 1.0 / (h * h);
    for (int k = 1; k < nz - 1; k++)
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) {
                if (((i + j + k) & 1) != color) continue;
                size_t p = at(nx, ny, i, j, k);
                double off = 0.0;
                for (int n = 0; n < 6; n++) {
                    int a = i + NB[n][0], b = j + NB[n][1], c = k + NB[n][2];
                    off += orc_face(D[p], D[at(nx, ny, a, b, c)], harmonic) * ih2 *
                           val0(nx, ny, nz, u, a, b, c);
                }
                u[p] = (f[p] + off) / diag_at(nx, ny, h, harmonic, D, mu, i, j, k);
            }
}

/*
 * Transpose of orc_gs_half acting on cotangents (Eqs. 10-11 in 3D):
 * for every p of the colour, t = ubar_p / diag_p; fbar_p += t;
 * ubar_j += a_pj t for each interior neighbour j; ubar_p = 0.
 */
static void gs_half_T(int nx, int ny, int nz, double h, int harmonic, const double *D,
                      const double *mu, double *ubar, double *fbar, int color) {
    double ih2 = 1.0 / (h * h);
    for (int k = 1; k < nz - 1; k++)
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) {
                if (((i + j + k) & 1) != color) continue;
                size_t p = at(nx, ny, i, j, k);
                double t = ubar[p] / diag_at(nx, ny, h, harmonic, D, mu, i, j, k);
                fbar[p] += t;
                for (int n = 0; n < 6; n++) {
                    int a = i + NB[n][0], b = j + NB[n][1], c = k + NB[n][2];
                    if (!is_interior(nx, ny, nz, a, b, c)) continue;
                    ubar[at(nx, ny, a, b, c)] +=
                        orc_face(D[p], D[at(nx, ny, a, b, c)], harmonic) * ih2 * t;
                }
                ubar[p] = 0.0;
            }
}

/* 1/4 [1 2 1] weight of an offset in {-1,0,1} (Eq. 7) */
static double fw(int o) { return o == 0 ? 0.5 : 0.25; }

/*
 * Full-weighting restriction (Eq. 7, tensor product in 3D) of a fine field
 * that is zero on the fine boundary, onto coarse interior vertices.
 */
void orc_restrict(int nxf, int nyf, int nzf, const double *r, double *fc) {
    int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1, nzc = (nzf - 1) / 2 + 1;
    for (int K = 0; K < nzc; K++)
        for (int J = 0; J < nyc; J++)
            for (int I = 0; I < nxc; I++) {
                double s = 0.0;
                if (is_interior(nxc, nyc, nzc, I, J, K))
                    for (int c = -1; c <= 1; c++)
                        for (int b = -1; b <= 1; b++)
                            for (int a = -1; a <= 1; a++)
                                s += fw(a) * fw(b) * fw(c) *
                                     r[at(nxf, nyf, 2 * I + a, 2 * J + b, 2 * K + c)];
                fc[at(nxc, nyc, I, J, K)] = s;
            }
}

/*
 * Prolongation I = 2^3 R^T (Eq. 17): every coarse interior value is spread to
 * the 27 fine vertices around 2I with weight 8 * 1/4[1 2 1]^3, i.e. trilinear
 * interpolation. out_fine += I e_coarse on fine interior vertices.
 */
void orc_prolong_add(int nxc, int nyc, int nzc, const double *e, double *uf) {
    int nxf = 2 * (nxc - 1) + 1, nyf = 2 * (nyc - 1) + 1, nzf = 2 * (nzc - 1) + 1;
    for (int K = 1; K < nzc - 1; K++)
        for (int J = 1; J < nyc - 1; J++)
            for (int I = 1; I < nxc - 1; I++) {
                double v = e[at(nxc, nyc, I, J, K)];
                for (int c = -1; c <= 1; c++)
                    for (int b = -1; b <= 1; b++)
                        for (int a = -1; a <= 1; a++) {
                            int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
                            if (!is_interior(nxf, nyf, nzf, i, j, k)) continue;
                            uf[at(nxf, nyf, i, j, k)] += 8.0 * fw(a) * fw(b) * fw(c) * v;
                        }
            }
}

/*
 * Coefficient coarsening for the rediscretised coarse operator L^{k+1}
 * (Sec. 2.2 states rediscretisation, not the rule): full weighting of the
 * vertex field on coarse interior vertices, injection on the coarse boundary;
 * inject != 0 selects injection everywhere.
 */
void orc_coarsen(int nxf, int nyf, int nzf, int inject, const double *Xf, double *Xc) {
    int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1, nzc = (nzf - 1) / 2 + 1;
    for (int K = 0; K < nzc; K++)
        for (int J = 0; J < nyc; J++)
            for (int I = 0; I < nxc; I++) {
                double s;
                if (inject || !is_interior(nxc, nyc, nzc, I, J, K)) {
                    s = Xf[at(nxf, nyf, 2 * I, 2 * J, 2 * K)];
                } else {
                    s = 0.0;
                    for (int c = -1; c <= 1; c++)
                        for (int b = -1; b <= 1; b++)
                            for (int a = -1; a <= 1; a++)
                                s += fw(a) * fw(b) * fw(c) *
                                     Xf[at(nxf, nyf, 2 * I + a, 2 * J + b, 2 * K + c)];
                }
                Xc[at(nxc, nyc, I, J, K)] = s;
            }
}

/* ------------------------------------------------------------------------ */
/* hierarchy                                                                 */

typedef struct {
    int nx, ny, nz;
    double h;
    double *D, *mu, *u, *f, *r;   /* vertex arrays */
    double *ub, *fb;              /* cotangents (literal adjoint) */
} orc_level;

typedef struct {
    int nlev, harmonic, inject, nu1, nu2, symmetric;
    orc_level L[ORC_MAXLEV];
    int nc;                /* coarsest interior unknowns */
    int *cidx;             /* coarsest interior -> vertex index */
    double *chol;          /* nc x nc lower Cholesky factor of L^{coarsest} */
} orc_h;

static size_t npts(const orc_level *l) { return (size_t)l->nx * l->ny * l->nz; }

/* number of levels: halve while every axis has an odd count > 3 */
int orc_count_levels(int nx, int ny, int nz) {
    if (nx < 3 || ny < 3 || nz < 3) return 0;
    int n = 1;
    while (nx > 3 && ny > 3 && nz > 3 && (nx - 1) % 2 == 0 && (ny - 1) % 2 == 0 &&
           (nz - 1) % 2 == 0) {
        nx = (nx - 1) / 2 + 1; ny = (ny - 1) / 2 + 1; nz = (nz - 1) / 2 + 1;
        n++;
        if (n > ORC_MAXLEV) return 0;
    }
    return n;
}

static int chol_factor(int n, double *a) {
    for (int j = 0; j < n; j++) {
        double s = a[(size_t)j * n + j];
        for (int k = 0; k < j; k++) s -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
        if (!(s > 0.0)) return -1;
        double d = sqrt(s);
        a[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double t = a[(size_t)i * n + j];
            for (int k = 0; k < j; k++) t -= a[(size_t)i * n + k] * a[(size_t)j * n + k];
            a[(size_t)i * n + j] = t / d;
        }
        for (int i = 0; i < j; i++) a[(size_t)i * n + j] = 0.0;
    }
    return 0;
}

static void chol_solve(int n, const double *l, double *x) {
    for (int i = 0; i < n; i++) {
        double t = x[i];
        for (int k = 0; k < i; k++) t -= l[(size_t)i * n + k] * x[k];
        x[i] = t / l[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double t = x[i];
        for (int k = i + 1; k < n; k++) t -= l[(size_t)k * n + i] * x[k];
        x[i] = t / l[(size_t)i * n + i];
    }
}

void orc_free(orc_h *H) {
    if (!H) return;
    for (int l = 0; l < H->nlev; l++) {
        orc_level *L = &H->L[l];
        free(L->D); free(L->mu); free(L->u); free(L->f); free(L->r);
        free(L->ub); free(L->fb);
    }
    free(H->cidx); free(H->chol); free(H);
}

/*
 * Build the hierarchy: coarse coefficients level by level, and the exact
 * coarsest solve, whose matrix is assembled column by column by applying the
 * coarsest operator to unit vectors. Returns NULL on invalid sizes or a
 * non-SPD coarsest matrix.
 */
orc_h *orc_create(int nx, int ny, int nz, double h, int harmonic, int inject, int nu1,
                  int nu2, int symmetric, const double *D, const double *mu) {
    int nlev = orc_count_levels(nx, ny, nz);
    if (nlev == 0) return NULL;
    orc_h *H = (orc_h *)calloc(1, sizeof(orc_h));
    H->nlev = nlev; H->harmonic = harmonic; H->inject = inject;
    H->nu1 = nu1; H->nu2 = nu2; H->symmetric = symmetric;
    for (int l = 0; l < nlev; l++) {
        orc_level *L = &H->L[l];
        if (l == 0) { L->nx = nx; L->ny = ny; L->nz = nz; L->h = h; }
        else {
            L->nx = (H->L[l - 1].nx - 1) / 2 + 1; L->ny = (H->L[l - 1].ny - 1) / 2 + 1;
            L->nz = (H->L[l - 1].nz - 1) / 2 + 1; L->h = 2.0 * H->L[l - 1].h;
        }
        size_t n = npts(L);
        L->D = (double *)calloc(n, sizeof(double)); L->mu = (double *)calloc(n, sizeof(double));
        L->u = (double *)calloc(n, sizeof(double)); L->f = (double *)calloc(n, sizeof(double));
        L->r = (double *)calloc(n, sizeof(double));
        L->ub = (double *)calloc(n, sizeof(double)); L->fb = (double *)calloc(n, sizeof(double));
        if (l == 0) {
            memcpy(L->D, D, n * sizeof(double));
            memcpy(L->mu, mu, n * sizeof(double));
        } else {
            orc_level *F = &H->L[l - 1];
            orc_coarsen(F->nx, F->ny, F->nz, inject, F->D, L->D);
            orc_coarsen(F->nx, F->ny, F->nz, inject, F->mu, L->mu);
        }
    }
    orc_level *C = &H->L[nlev - 1];
    int nc = (C->nx - 2) * (C->ny - 2) * (C->nz - 2);
    H->nc = nc;
    H->cidx = (int *)malloc(sizeof(int) * nc);
    H->chol = (double *)calloc((size_t)nc * nc, sizeof(double));
    int q = 0;
    for (int k = 1; k < C->nz - 1; k++)
        for (int j = 1; j < C->ny - 1; j++)
            for (int i = 1; i < C->nx - 1; i++) H->cidx[q++] = (int)at(C->nx, C->ny, i, j, k);
    size_t n = npts(C);
    double *e = (double *)calloc(n, sizeof(double)), *ae = (double *)calloc(n, sizeof(double));
    for (int c = 0; c < nc; c++) {
        memset(e, 0, n * sizeof(double));
        e[H->cidx[c]] = 1.0;
        orc_apply(C->nx, C->ny, C->nz, C->h, harmonic, C->D, C->mu, e, ae);
        for (int r = 0; r < nc; r++) H->chol[(size_t)r * nc + c] = ae[H->cidx[r]];
    }
    free(e); free(ae);
    if (chol_factor(nc, H->chol) != 0) { orc_free(H); return NULL; }
    return H;
}

int orc_levels(const orc_h *H) { return H->nlev; }

void orc_level_dims(const orc_h *H, int l, int *dims) {
    dims[0] = H->L[l].nx; dims[1] = H->L[l].ny; dims[2] = H->L[l].nz;
}

void orc_level_coeffs(const orc_h *H, int l, double *D, double *mu) {
    size_t n = npts(&H->L[l]);
    if (D) memcpy(D, H->L[l].D, n * sizeof(double));
    if (mu) memcpy(mu, H->L[l].mu, n * sizeof(double));
}

static void coarsest_solve(orc_h *H, const double *f, double *u) {
    double *x = (double *)malloc(sizeof(double) * (size_t)H->nc);
    for (int c = 0; c < H->nc; c++) x[c] = f[H->cidx[c]];
    chol_solve(H->nc, H->chol, x);
    for (int c = 0; c < H->nc; c++) u[H->cidx[c]] = x[c];
    free(x);
}

static void sweep(orc_h *H, int l, int first) {
    orc_level *L = &H->L[l];
    orc_gs_half(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, L->f, L->u, first);
    orc_gs_half(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, L->f, L->u, 1 - first);
}

/*
 * One V-cycle at level l on (L->u, L->f) in place (Sec. 2.2, Fig. 1 left):
 * pre-smoothing, defect, restriction, zero coarse guess (Sec. 2.3.1, coarse
 * levels start at zero), recursion, prolongation and correction,
 * post-smoothing. transposed != 0 runs the V-cycle whose preconditioner is
 * the transpose of the forward one: nu2 pre sweeps and nu1 post sweeps, each
 * with the colour order reversed.
 *   forward:    pre  = nu1 x (red, black); post = nu2 x (red, black), or
 *               (black, red) when symmetric
 *   transposed: pre  = nu2 x reverse(post order); post = nu1 x (black, red)
 */
static void vcycle(orc_h *H, int l, int transposed) {
    orc_level *L = &H->L[l];
    if (l == H->nlev - 1) { coarsest_solve(H, L->f, L->u); return; }
    int post_first = H->symmetric ? 1 : 0;
    int npre = transposed ? H->nu2 : H->nu1, npost = transposed ? H->nu1 : H->nu2;
    int pre_first = transposed ? 1 - post_first : 0;
    int postf = transposed ? 1 : post_first;
    for (int s = 0; s < npre; s++) sweep(H, l, pre_first);
    orc_level *C = &H->L[l + 1];
    orc_residual(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, L->f, L->u, L->r);
    orc_restrict(L->nx, L->ny, L->nz, L->r, C->f);
    memset(C->u, 0, npts(C) * sizeof(double));
    vcycle(H, l + 1, transposed);
    orc_prolong_add(C->nx, C->ny, C->nz, C->u, L->u);
    for (int s = 0; s < npost; s++) sweep(H, l, postf);
}

static double norm_int(int nx, int ny, int nz, const double *x) {
    double s = 0.0;
    for (int k = 1; k < nz - 1; k++)
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) {
                double v = x[at(nx, ny, i, j, k)];
                s += v * v;
            }
    return sqrt(s);
}

/* ||f - A u||_2 / ||f||_2 over interior vertices at level 0 */
double orc_rel_residual(orc_h *H, const double *f, const double *u) {
    orc_level *L = &H->L[0];
    double *r = (double *)calloc(npts(L), sizeof(double));
    orc_residual(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, f, u, r);
    double nr = norm_int(L->nx, L->ny, L->nz, r), nf = norm_int(L->nx, L->ny, L->nz, f);
    free(r);
    return nf > 0.0 ? nr / nf : nr;
}

/*
 * Iterate V-cycles from u = 0 on A u = rhs (the solver S of Eq. 2/Eq. 5).
 * fixed > 0: exactly that many cycles (the paper's fixed-count mode, Sec. 2.4).
 * fixed == 0: until ||rhs - A u|| <= rtol ||rhs|| or max_cycles.
 * hist (may be NULL) receives the relative residual after every cycle (up to
 * hist_len entries). Returns the number of cycles run.
 */
static int iterate(orc_h *H, const double *rhs, double *out, double rtol, int max_cycles,
                   int fixed, double *hist, int hist_len, int transposed) {
    orc_level *L = &H->L[0];
    size_t n = npts(L);
    for (int k = 0; k < L->nz; k++)
        for (int j = 0; j < L->ny; j++)
            for (int i = 0; i < L->nx; i++) {
                size_t p = at(L->nx, L->ny, i, j, k);
                L->f[p] = is_interior(L->nx, L->ny, L->nz, i, j, k) ? rhs[p] : 0.0;
            }
    memset(L->u, 0, n * sizeof(double));
    int ncyc = fixed > 0 ? fixed : max_cycles;
    int c = 0;
    double nf = norm_int(L->nx, L->ny, L->nz, L->f);
    if (fixed == 0 && nf == 0.0) { memcpy(out, L->u, n * sizeof(double)); return 0; }
    for (c = 1; c <= ncyc; c++) {
        vcycle(H, 0, transposed);
        if (fixed == 0 || hist) {
            double rel = orc_rel_residual(H, L->f, L->u);
            if (hist && c - 1 < hist_len) hist[c - 1] = rel;
            if (fixed == 0 && rel <= rtol) break;
        }
    }
    if (c > ncyc) c = ncyc;
    memcpy(out, L->u, n * sizeof(double));
    return c;
}

int orc_solve(orc_h *H, const double *q, double *u, double rtol, int max_cycles, int fixed,
              double *hist, int hist_len) {
    return iterate(H, q, u, rtol, max_cycles, fixed, hist, hist_len, 0);
}

/*
 * Adjoint solve lambda = S_m^T w by the transposed V-cycle iteration: with
 * S_m = sum_{c<m} (I - B A)^c B, S_m^T = sum_{c<m} (I - B^T A)^c B^T because
 * A is symmetric, i.e. m cycles of the transposed V-cycle from zero.
 * fixed == 0 iterates to rtol instead (the converged adjoint A^{-1} w).
 */
int orc_adjoint(orc_h *H, const double *w, double *lam, double rtol, int max_cycles,
                int fixed, double *hist, int hist_len) {
    return iterate(H, w, lam, rtol, max_cycles, fixed, hist, hist_len, 1);
}

/* apply one V-cycle at level 0 in place: u <- V(u, f) */
void orc_vcycle(orc_h *H, const double *f, double *u, int transposed) {
    orc_level *L = &H->L[0];
    size_t n = npts(L);
    memcpy(L->f, f, n * sizeof(double));
    memcpy(L->u, u, n * sizeof(double));
    vcycle(H, 0, transposed);
    memcpy(u, L->u, n * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* literal reversed composition (Sec. 2.4, Eq. 18; Fig. 1 right)            */

static void rev_vcycle(orc_h *H, int l) {
    orc_level *L = &H->L[l];
    size_t n = npts(L);
    if (l == H->nlev - 1) {
        /* forward: u_L = A_L^{-1} f_L (u_L overwritten) */
        double *t = (double *)calloc(n, sizeof(double));
        coarsest_solve(H, L->ub, t);
        for (size_t p = 0; p < n; p++) { L->fb[p] += t[p]; L->ub[p] = 0.0; }
        free(t);
        return;
    }
    orc_level *C = &H->L[l + 1];
    size_t nc = npts(C);
    int post_first = H->symmetric ? 1 : 0;
    /* post-smoothing, last half-sweep first */
    for (int s = 0; s < H->nu2; s++) {
        gs_half_T(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, L->ub, L->fb,
                  1 - post_first);
        gs_half_T(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, L->ub, L->fb,
                  post_first);
    }
    /* u_l += I u_{l+1}  ->  ubar_{l+1} += I^T ubar_l = 2^3 R ubar_l (Sec. 2.3.3) */
    double *t = (double *)calloc(nc, sizeof(double));
    orc_restrict(L->nx, L->ny, L->nz, L->ub, t);
    for (size_t p = 0; p < nc; p++) C->ub[p] += 8.0 * t[p];
    free(t);
    rev_vcycle(H, l + 1);
    /* u_{l+1} = 0  ->  its cotangent is dropped */
    memset(C->ub, 0, nc * sizeof(double));
    /* f_{l+1} = R (f_l - A_l u_l)  ->  fbar_l += R^T fbar_{l+1},
       ubar_l -= A_l R^T fbar_{l+1}, fbar_{l+1} = 0 (Eqs. 15-16, R^T = 2^-3 I) */
    double *rt = (double *)calloc(n, sizeof(double));
    double *art = (double *)calloc(n, sizeof(double));
    orc_prolong_add(C->nx, C->ny, C->nz, C->fb, rt);
    for (size_t p = 0; p < n; p++) rt[p] *= 0.125;
    orc_apply(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, rt, art);
    for (size_t p = 0; p < n; p++) { L->fb[p] += rt[p]; L->ub[p] -= art[p]; }
    memset(C->fb, 0, nc * sizeof(double));
    free(rt); free(art);
    /* pre-smoothing, last half-sweep first */
    for (int s = 0; s < H->nu1; s++) {
        gs_half_T(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, L->ub, L->fb, 1);
        gs_half_T(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, L->ub, L->fb, 0);
    }
}

/*
 * qbar = S_m^dagger w computed as the reverse of the forward program: the
 * forward sets f_0 = q, u_0 = 0 and runs m V-cycles; the reverse seeds
 * ubar_0 = w, runs the m V-cycles' adjoints in reverse, and returns fbar_0.
 */
void orc_adjoint_literal(orc_h *H, const double *w, double *qbar, int m) {
    for (int l = 0; l < H->nlev; l++) {
        memset(H->L[l].ub, 0, npts(&H->L[l]) * sizeof(double));
        memset(H->L[l].fb, 0, npts(&H->L[l]) * sizeof(double));
    }
    orc_level *L = &H->L[0];
    for (int k = 0; k < L->nz; k++)
        for (int j = 0; j < L->ny; j++)
            for (int i = 0; i < L->nx; i++) {
                size_t p = at(L->nx, L->ny, i, j, k);
                L->ub[p] = is_interior(L->nx, L->ny, L->nz, i, j, k) ? w[p] : 0.0;
            }
    for (int c = 0; c < m; c++) rev_vcycle(H, 0);
    for (int k = 0; k < L->nz; k++)
        for (int j = 0; j < L->ny; j++)
            for (int i = 0; i < L->nx; i++) {
                size_t p = at(L->nx, L->ny, i, j, k);
                qbar[p] = is_interior(L->nx, L->ny, L->nz, i, j, k) ? L->fb[p] : 0.0;
            }
}

/* ------------------------------------------------------------------------ */
/* coefficient derivatives                                                   */

/*
 * Gradients of <w, u> through A(D, mu) u = q given u and the adjoint state
 * lambda = A^{-T} w: d<w,u> = -lambda^T (dA) u.
 *   mubar_p = -lambda_p u_p on interior p, 0 on the boundary
 *   Dbar_v  = -(1/h^2) sum_{j in nbr(v)} dface(D_v, D_j)/dD_v
 *             (lambda_v - lambda_j)(u_v - u_j),  u, lambda = 0 off the interior
 * Dbar is defined on every vertex, boundary vertices included.
 */
void orc_grad(int nx, int ny, int nz, double h, int harmonic, const double *D,
              const double *u, const double *lam, double *Dbar, double *mubar) {
    double ih2 = 1.0 / (h * h);
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t p = at(nx, ny, i, j, k);
                double uv = val0(nx, ny, nz, u, i, j, k), lv = val0(nx, ny, nz, lam, i, j, k);
                mubar[p] = -lv * uv;
                double s = 0.0;
                for (int n = 0; n < 6; n++) {
                    int a = i + NB[n][0], b = j + NB[n][1], c = k + NB[n][2];
                    if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
                    double uj = val0(nx, ny, nz, u, a, b, c), lj = val0(nx, ny, nz, lam, a, b, c);
                    s += orc_face_da(D[p], D[at(nx, ny, a, b, c)], harmonic) * (lv - lj) * (uv - uj);
                }
                Dbar[p] = -s * ih2;
            }
}

/*
 * out = (dA) u for tangents dD (every vertex) and dmu: the derivative of the
 * operator of Eq. 1 in the direction (dD, dmu), interior only.
 */
void orc_dA_apply(int nx, int ny, int nz, double h, int harmonic, const double *D,
                  const double *dD, const double *dmu, const double *u, double *out) {
    double ih2 = 1.0 / (h * h);
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t p = at(nx, ny, i, j, k);
                if (!is_interior(nx, ny, nz, i, j, k)) { out[p] = 0.0; continue; }
                double s = 0.0;
                for (int n = 0; n < 6; n++) {
                    int a = i + NB[n][0], b = j + NB[n][1], c = k + NB[n][2];
                    size_t q = at(nx, ny, a, b, c);
                    double dface = dD ? orc_face_da(D[p], D[q], harmonic) * dD[p] +
                                            orc_face_da(D[q], D[p], harmonic) * dD[q]
                                      : 0.0;
                    s += dface * (u[p] - val0(nx, ny, nz, u, a, b, c));
                }
                out[p] = s * ih2 + (dmu ? dmu[p] : 0.0) * u[p];
            }
}
