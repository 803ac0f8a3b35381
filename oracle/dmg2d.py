"""FP64 oracle of the two-dimensional solver: the same method as the 3D oracle
(arXiv 2608.00760, Sec. 2.2-2.4) on a (ny, nx) vertex grid, where the paper
runs its 2D benchmarks (Sec. 3).

TEST INFRASTRUCTURE: only tests/ may use it; it shares no code with the CUDA
path.

Definitions (each the 2D reading of the 3D oracle's):
- operator (Eq. 1, 5-point): (A u)_p = (1/h^2) sum_{j in nbr(p)} face(D_p, D_j)(u_p - u_j)
  + mu_p u_p on interior vertices, u = 0 on the boundary (Dirichlet);
  face = arithmetic mean (or harmonic);
- red-black Gauss-Seidel (Eq. 9), red = even i + j, updated first;
- full weighting R = 1/4 [1 2 1] per axis (Eq. 7), prolongation P = 2^2 R^T
  (Eq. 17, bilinear interpolation);
- coarse coefficients: full weighting on coarse interior vertices, injection on
  the coarse boundary; coarsest level solved exactly;
- V-cycle: nu1 pre-sweeps, defect, restriction, zero coarse guess, recursion,
  prolongation, nu2 post-sweeps; the transposed cycle runs nu2 pre-sweeps and
  nu1 post-sweeps with the colour orders reversed (Sec. 2.4);
- gradients of <w, u>: Dbar_v = -(1/h^2) sum_{j nbr v} dface/dD_v (lam_v - lam_j)(u_v - u_j),
  mubar_v = -lam_v u_v, with lam = A^{-1} w (adjoint state).

Parity status: pinned. tests/test_oracle_2d.py checks the operator on the
discrete eigenfunctions (closed form), symmetry, the multigrid solve against a
library sparse direct solve, P = 4 R^T by brute force, the transposed cycle as
the exact transpose of the m-cycle solver, and the gradients by central finite
differences.
"""
from __future__ import annotations

import numpy as np

DIRS = ((-1, 0), (1, 0), (0, -1), (0, 1))   # (dx, dy)
_FW = {-1: 0.25, 0: 0.5, 1: 0.25}


def _face(a, b, harmonic):
    return 2.0 * a * b / (a + b) if harmonic else 0.5 * (a + b)


def _face_da(a, b, harmonic):
    return 2.0 * b * b / ((a + b) * (a + b)) if harmonic else 0.5 + 0.0 * a


def _sh(x, dx, dy):
    ny, nx = x.shape
    return x[1 + dy:ny - 1 + dy, 1 + dx:nx - 1 + dx]


def _colour(shape):
    ny, nx = shape
    j, i = np.meshgrid(np.arange(1, ny - 1), np.arange(1, nx - 1), indexing="ij")
    return (i + j) & 1


def _zero_boundary(x):
    x = x.copy()
    x[0, :] = x[-1, :] = 0
    x[:, 0] = x[:, -1] = 0
    return x


def apply(D, mu, h, u, harmonic=False):
    out = np.zeros_like(u)
    c, uc = _sh(D, 0, 0), _sh(u, 0, 0)
    s = 0.0
    for dx, dy in DIRS:
        s = s + _face(c, _sh(D, dx, dy), harmonic) * (uc - _sh(u, dx, dy))
    out[1:-1, 1:-1] = s / (h * h) + _sh(mu, 0, 0) * uc
    return out


def gs_half(D, mu, h, f, u, colour, harmonic=False):
    c = _sh(D, 0, 0)
    off, dg = 0.0, 0.0
    for dx, dy in DIRS:
        a = _face(c, _sh(D, dx, dy), harmonic) / (h * h)
        off = off + a * _sh(u, dx, dy)
        dg = dg + a
    new = (_sh(f, 0, 0) + off) / (dg + _sh(mu, 0, 0))
    inner = u[1:-1, 1:-1]
    sel = _colour(u.shape) == colour
    inner[sel] = new[sel]


def _coarse(n):
    return (n - 1) // 2 + 1


def restrict(r):
    ny, nx = r.shape
    Jc, Ic = _coarse(ny), _coarse(nx)
    out = np.zeros((Jc, Ic), dtype=r.dtype)
    s = 0.0
    for b in (-1, 0, 1):
        for a in (-1, 0, 1):
            s = s + _FW[a] * _FW[b] * r[2 + b:2 * (Jc - 1) + b:2, 2 + a:2 * (Ic - 1) + a:2]
    out[1:-1, 1:-1] = s
    return out


def prolong_add(e, uf):
    Jc, Ic = e.shape
    ec = e[1:-1, 1:-1]
    acc = np.zeros_like(uf)
    for b in (-1, 0, 1):
        for a in (-1, 0, 1):
            acc[2 + b:2 * (Jc - 1) + b:2, 2 + a:2 * (Ic - 1) + a:2] += 4.0 * _FW[a] * _FW[b] * ec
    uf[1:-1, 1:-1] += acc[1:-1, 1:-1]


def coarsen(X, inject=False):
    out = X[::2, ::2].copy()
    if not inject:
        out[1:-1, 1:-1] = restrict(X)[1:-1, 1:-1]
    return out


def count_levels(shape):
    n, s = 1, list(shape)
    while all(x > 3 and (x - 1) % 2 == 0 for x in s):
        s = [_coarse(x) for x in s]
        n += 1
    return n


def interior_index(shape):
    return np.flatnonzero(np.pad(np.ones(tuple(x - 2 for x in shape), dtype=bool), 1))


def assemble(D, mu, h, harmonic=False):
    """Sparse A on interior unknowns, column by column from `apply` on unit vectors."""
    import scipy.sparse as sp
    idx = interior_index(D.shape)
    cols = []
    e = np.zeros(D.shape)
    for c in range(idx.size):
        e.reshape(-1)[idx[c]] = 1.0
        cols.append(sp.csc_matrix(apply(D, mu, h, e, harmonic).reshape(-1)[idx][:, None]))
        e.reshape(-1)[idx[c]] = 0.0
    return sp.hstack(cols).tocsr(), idx


def direct_solve(D, mu, h, q, harmonic=False):
    import scipy.sparse.linalg as spla
    A, idx = assemble(D, mu, h, harmonic)
    u = np.zeros(D.shape)
    u.reshape(-1)[idx] = spla.spsolve(A.tocsc(), np.asarray(q).reshape(-1)[idx])
    return u


class Hierarchy:
    """Levels, the exact coarsest solve, the V-cycle and its transpose (2D)."""

    def __init__(self, D, mu, h, nu1=2, nu2=2, harmonic=False, inject=False, symmetric=False):
        self.D, self.mu, self.h = np.asarray(D, float), np.asarray(mu, float), float(h)
        self.shape = self.D.shape
        self.nu1, self.nu2, self.harmonic, self.symmetric = nu1, nu2, harmonic, symmetric
        self.levels = [(self.D, self.mu, self.h)]
        for _ in range(count_levels(self.shape) - 1):
            Dp, mp, hp = self.levels[-1]
            self.levels.append((coarsen(Dp, inject), coarsen(mp, inject), 2.0 * hp))
        Dc, mc, hc = self.levels[-1]
        A, self.cidx = assemble(Dc, mc, hc, harmonic)
        self.Ainv = np.linalg.inv(A.toarray())

    def vcycle(self, l, f, u, transposed=False):
        D, mu, h = self.levels[l]
        if l == len(self.levels) - 1:
            u.reshape(-1)[self.cidx] = self.Ainv @ f.reshape(-1)[self.cidx]
            return
        post_first = 1 if self.symmetric else 0
        npre, npost = (self.nu2, self.nu1) if transposed else (self.nu1, self.nu2)
        pre_first = 1 - post_first if transposed else 0
        postf = 1 if transposed else post_first
        for _ in range(npre):
            gs_half(D, mu, h, f, u, pre_first, self.harmonic)
            gs_half(D, mu, h, f, u, 1 - pre_first, self.harmonic)
        r = _zero_boundary(f - apply(D, mu, h, u, self.harmonic))
        fc = restrict(r)
        uc = np.zeros_like(fc)
        self.vcycle(l + 1, fc, uc, transposed)
        prolong_add(uc, u)
        for _ in range(npost):
            gs_half(D, mu, h, f, u, postf, self.harmonic)
            gs_half(D, mu, h, f, u, 1 - postf, self.harmonic)

    def rel_residual(self, f, u):
        r = _zero_boundary(f - apply(self.D, self.mu, self.h, u, self.harmonic))
        fi = _zero_boundary(f)
        return np.linalg.norm(r) / np.linalg.norm(fi)

    def _iterate(self, rhs, rtol, max_cycles, fixed, transposed):
        f = _zero_boundary(np.asarray(rhs, float))
        u = np.zeros_like(f)
        nf = np.linalg.norm(f)
        if nf == 0.0:
            return u, 0
        cycles = fixed if fixed > 0 else max_cycles
        for c in range(1, cycles + 1):
            self.vcycle(0, f, u, transposed)
            if fixed == 0 and self.rel_residual(f, u) <= rtol:
                return u, c
        return u, cycles

    def solve(self, q, rtol=1e-10, max_cycles=100, fixed=0):
        return self._iterate(q, rtol, max_cycles, fixed, False)

    def adjoint(self, w, rtol=1e-10, max_cycles=100, fixed=0):
        return self._iterate(w, rtol, max_cycles, fixed, True)

    def vjp(self, u, w, rtol=1e-10, max_cycles=100, fixed=0):
        lam, c = self.adjoint(w, rtol=rtol, max_cycles=max_cycles, fixed=fixed)
        Db, mb = grad(self.D, self.h, u, lam, self.harmonic)
        return lam, Db, mb, c

    def jvp(self, u, dq, dD=None, dmu=None, rtol=1e-10, max_cycles=100, fixed=0):
        rhs = np.asarray(dq, float).copy()
        if dD is not None or dmu is not None:
            rhs = rhs - dA_apply(self.D, self.h, dD, dmu, u, self.harmonic)
        return self.solve(rhs, rtol=rtol, max_cycles=max_cycles, fixed=fixed)


def grad(D, h, u, lam, harmonic=False):
    """(Dbar, mubar) of <w, u> from u and lam = A^{-1} w (every vertex; u, lam zero on the boundary)."""
    ny, nx = D.shape
    Db = np.zeros_like(D)
    for dx, dy in DIRS:
        # contribution of the face between v and v + (dx, dy) to Dbar_v
        js = slice(max(0, -dy), ny - max(0, dy))
        is_ = slice(max(0, -dx), nx - max(0, dx))
        jn = slice(max(0, dy), ny - max(0, -dy))
        in_ = slice(max(0, dx), nx - max(0, -dx))
        Dv, Dn = D[js, is_], D[jn, in_]
        Db[js, is_] += _face_da(Dv, Dn, harmonic) * (lam[js, is_] - lam[jn, in_]) * (u[js, is_] - u[jn, in_])
    Db = -Db / (h * h)
    mb = _zero_boundary(-lam * u)
    return Db, mb


def dA_apply(D, h, dD, dmu, u, harmonic=False):
    """(dA) u on interior vertices for a coefficient direction (dD, dmu)."""
    out = np.zeros_like(u)
    c, uc = _sh(D, 0, 0), _sh(u, 0, 0)
    s = 0.0
    if dD is not None:
        dc = _sh(dD, 0, 0)
        for dx, dy in DIRS:
            Dn, dn = _sh(D, dx, dy), _sh(dD, dx, dy)
            dface = _face_da(c, Dn, harmonic) * dc + _face_da(Dn, c, harmonic) * dn
            s = s + dface * (uc - _sh(u, dx, dy))
    s = s / (h * h)
    if dmu is not None:
        s = s + _sh(dmu, 0, 0) * uc
    out[1:-1, 1:-1] = s
    return out
