"""Oracle for the unrolled coefficient gradient: the exact derivative of the
fixed-count solver S_m(q; D, mu) (m V-cycles from u = 0, Sec. 2.2) with respect
to q, D and mu, through every iterate and through the coarsened coefficients of
every level.

TEST INFRASTRUCTURE (see the package header): only tests may use it.

The derivative is taken by the complex step: for a map F that is analytic in
its real inputs, dF(x)[d] = Im F(x + i e d) / e for a tiny e (1e-30 here), with
no subtractive cancellation, so it is exact to rounding. The V-cycle below is
written once in numpy for any dtype, following the same definitions as the C
oracle (dmg_oracle.c): the 7-point operator with face means (Eq. 1), red-black
Gauss-Seidel half-sweeps (Eq. 9, red = even i+j+k first), defect and full
weighting (Eqs. 7, 13), zero coarse guess, prolongation 2^3 R^T (Eq. 17), the
exact coarsest solve, and coefficient coarsening by full weighting inside and
injection on the boundary. Every step is analytic in D and mu (sums, products,
quotients, a linear solve), so S_m is too.

Parity status: pinned. tests/test_oracle_unrolled.py checks the real V-cycle
against the C oracle's fixed-cycle solve, and the complex-step derivatives
against central finite differences of the C oracle's fixed-cycle solve.
"""
from __future__ import annotations

import numpy as np

DIRS = ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))   # (dx, dy, dz)


def _face(a, b, harmonic):
    return 2.0 * a * b / (a + b) if harmonic else 0.5 * (a + b)


def _shift(x, dx, dy, dz):
    """y[k, j, i] = x[k + dz, j + dy, i + dx] on interior vertices (views of the interior box)."""
    nz, ny, nx = x.shape
    return x[1 + dz:nz - 1 + dz, 1 + dy:ny - 1 + dy, 1 + dx:nx - 1 + dx]


def _colour(shape):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(1, nz - 1), np.arange(1, ny - 1), np.arange(1, nx - 1), indexing="ij")
    return (i + j + k) & 1


def apply(D, mu, h, u, harmonic=False):
    """A u on interior vertices (u zero on the boundary), zero on the boundary."""
    out = np.zeros_like(u)
    c = _shift(D, 0, 0, 0)
    uc = _shift(u, 0, 0, 0)
    s = 0.0
    for dx, dy, dz in DIRS:
        s = s + _face(c, _shift(D, dx, dy, dz), harmonic) * (uc - _shift(u, dx, dy, dz))
    out[1:-1, 1:-1, 1:-1] = s / (h * h) + _shift(mu, 0, 0, 0) * uc
    return out


def gs_half(D, mu, h, f, u, colour, harmonic=False):
    """Red-black Gauss-Seidel on one colour, in place (Eq. 9)."""
    c = _shift(D, 0, 0, 0)
    off, dg = 0.0, 0.0
    for dx, dy, dz in DIRS:
        a = _face(c, _shift(D, dx, dy, dz), harmonic) / (h * h)
        off = off + a * _shift(u, dx, dy, dz)
        dg = dg + a
    new = (_shift(f, 0, 0, 0) + off) / (dg + _shift(mu, 0, 0, 0))
    inner = u[1:-1, 1:-1, 1:-1]
    sel = _colour(u.shape) == colour
    inner[sel] = new[sel]


_FW = {-1: 0.25, 0: 0.5, 1: 0.25}


def _coarse(n):
    return (n - 1) // 2 + 1


def restrict(r):
    """Full weighting onto coarse interior vertices (Eq. 7)."""
    nz, ny, nx = r.shape
    out = np.zeros((_coarse(nz), _coarse(ny), _coarse(nx)), dtype=r.dtype)
    Kc, Jc, Ic = out.shape
    s = 0.0
    for c in (-1, 0, 1):
        for b in (-1, 0, 1):
            for a in (-1, 0, 1):
                s = s + _FW[a] * _FW[b] * _FW[c] * r[2 + c:2 * (Kc - 1) + c:2, 2 + b:2 * (Jc - 1) + b:2,
                                                     2 + a:2 * (Ic - 1) + a:2]
    out[1:-1, 1:-1, 1:-1] = s
    return out


def prolong_add(e, uf):
    """uf += 2^3 R^T e on fine interior vertices (Eq. 17)."""
    Kc, Jc, Ic = e.shape
    ec = e[1:-1, 1:-1, 1:-1]
    acc = np.zeros_like(uf)
    for c in (-1, 0, 1):
        for b in (-1, 0, 1):
            for a in (-1, 0, 1):
                acc[2 + c:2 * (Kc - 1) + c:2, 2 + b:2 * (Jc - 1) + b:2, 2 + a:2 * (Ic - 1) + a:2] += (
                    8.0 * _FW[a] * _FW[b] * _FW[c] * ec)
    uf[1:-1, 1:-1, 1:-1] += acc[1:-1, 1:-1, 1:-1]


def coarsen(X, inject=False):
    """Coarse coefficients: full weighting on coarse interior vertices, injection on the coarse boundary."""
    out = X[::2, ::2, ::2].copy()
    if not inject:
        out[1:-1, 1:-1, 1:-1] = restrict(X)[1:-1, 1:-1, 1:-1]
    return out


def count_levels(shape):
    n = 1
    s = list(shape)
    while all(x > 3 and (x - 1) % 2 == 0 for x in s):
        s = [_coarse(x) for x in s]
        n += 1
    return n


class Hierarchy:
    """Levels (D_l, mu_l, h_l) and the dense coarsest operator, for any dtype."""

    def __init__(self, D, mu, h, nu1=2, nu2=2, harmonic=False, inject=False, symmetric=False):
        self.nu1, self.nu2, self.harmonic, self.symmetric = nu1, nu2, harmonic, symmetric
        self.levels = [(D, mu, float(h))]
        for _ in range(count_levels(D.shape) - 1):
            Dp, mp, hp = self.levels[-1]
            self.levels.append((coarsen(Dp, inject), coarsen(mp, inject), 2.0 * hp))
        Dc, mc, hc = self.levels[-1]
        shape = Dc.shape
        idx = np.flatnonzero(np.pad(np.ones(tuple(s - 2 for s in shape), dtype=bool), 1))
        n = idx.size
        Ac = np.zeros((n, n), dtype=np.result_type(D, mu))
        e = np.zeros(shape, dtype=Ac.dtype)
        for col in range(n):
            e.reshape(-1)[idx[col]] = 1.0
            Ac[:, col] = apply(Dc, mc, hc, e, harmonic).reshape(-1)[idx]
            e.reshape(-1)[idx[col]] = 0.0
        self.cidx, self.Ac = idx, Ac

    def vcycle(self, l, f, u):
        D, mu, h = self.levels[l]
        if l == len(self.levels) - 1:
            u.reshape(-1)[self.cidx] = np.linalg.solve(self.Ac, f.reshape(-1)[self.cidx])
            return
        post_first = 1 if self.symmetric else 0
        for _ in range(self.nu1):
            gs_half(D, mu, h, f, u, 0, self.harmonic)
            gs_half(D, mu, h, f, u, 1, self.harmonic)
        r = f - apply(D, mu, h, u, self.harmonic)
        r[0, :, :] = r[-1, :, :] = 0
        r[:, 0, :] = r[:, -1, :] = 0
        r[:, :, 0] = r[:, :, -1] = 0
        fc = restrict(r)
        uc = np.zeros_like(fc)
        self.vcycle(l + 1, fc, uc)
        prolong_add(uc, u)
        for _ in range(self.nu2):
            gs_half(D, mu, h, f, u, post_first, self.harmonic)
            gs_half(D, mu, h, f, u, 1 - post_first, self.harmonic)


def solve_fixed(D, mu, h, q, m, **kw):
    """S_m(q; D, mu): m V-cycles from u = 0 (q on boundary vertices ignored)."""
    H = Hierarchy(D, mu, h, **kw)
    f = np.array(q, dtype=np.result_type(D, mu, q))
    f[0, :, :] = f[-1, :, :] = 0
    f[:, 0, :] = f[:, -1, :] = 0
    f[:, :, 0] = f[:, :, -1] = 0
    u = np.zeros_like(f)
    for _ in range(m):
        H.vcycle(0, f, u)
    return u


def directional(D, mu, h, q, w, m, dq=None, dD=None, dmu=None, eps=1e-30, **kw):
    """d/dt <w, S_m(q + t dq; D + t dD, mu + t dmu)> at t = 0, by the complex step."""
    z = lambda x, d: x + 1j * eps * d if d is not None else x.astype(complex)
    u = solve_fixed(z(D, dD), z(mu, dmu), h, z(q, dq), m, **kw)
    return float(np.sum(w * u).imag / eps)


def gradient(D, mu, h, q, w, m, **kw):
    """(qbar, Dbar, mubar) of <w, S_m> entry by entry (one complex solve per
    vertex and field): small grids only."""
    out = []
    for which in ("q", "D", "mu"):
        g = np.zeros(D.shape)
        for p in range(D.size):
            d = np.zeros(D.shape)
            d.reshape(-1)[p] = 1.0
            kwd = {"dq": d} if which == "q" else ({"dD": d} if which == "D" else {"dmu": d})
            g.reshape(-1)[p] = directional(D, mu, h, q, w, m, **kwd, **kw)
        out.append(g)
    return tuple(out)
