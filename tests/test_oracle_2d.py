"""Pins of the 2D oracle (oracle/dmg2d.py): the 5-point operator on the discrete
eigenfunctions (closed form) and its symmetry, the multigrid solve against a
library sparse direct solve, P = 4 R^T by brute force, the transposed cycle as
the exact transpose of the m-cycle solver (matrices built column by column),
and the gradients and tangent against central finite differences."""
import numpy as np
import pytest

from oracle import dmg2d
from paper_2608_00760_b300 import inputs


def test_eigenfunctions_of_the_constant_operator():
    n, d, m = 17, 1.7, 0.3
    h = 1.0 / (n - 1)
    y, x = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="ij")
    D, mu = np.full((n, n), d), np.full((n, n), m)
    for p, q in ((1, 1), (2, 5), (7, 3)):
        u = np.sin(p * np.pi * x) * np.sin(q * np.pi * y)
        u[0, :] = u[-1, :] = u[:, 0] = u[:, -1] = 0.0
        lam = d * 4.0 / (h * h) * (np.sin(p * np.pi * h / 2) ** 2 + np.sin(q * np.pi * h / 2) ** 2) + m
        Au = dmg2d.apply(D, mu, h, u)
        assert np.abs(Au - lam * u).max() <= 1e-10 * lam


def test_operator_is_symmetric():
    w = inputs.tissue2d(seed=81, shape=(17, 33))
    rng = np.random.default_rng(1)
    u, v = (dmg2d._zero_boundary(rng.standard_normal(w["shape"])) for _ in range(2))
    for harm in (False, True):
        a = np.sum(v * dmg2d.apply(w["D"], w["mu"], w["h"], u, harm))
        b = np.sum(u * dmg2d.apply(w["D"], w["mu"], w["h"], v, harm))
        assert a == pytest.approx(b, rel=1e-13)


@pytest.mark.parametrize("shape", [(33, 33), (17, 65), (65, 129)])
def test_solve_matches_direct_solve(shape):
    w = inputs.tissue2d(seed=82, shape=shape)
    H = dmg2d.Hierarchy(w["D"], w["mu"], w["h"])
    u, c = H.solve(w["q"], rtol=1e-12)
    ref = dmg2d.direct_solve(w["D"], w["mu"], w["h"], w["q"])
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref) and c < 30


def test_prolongation_is_four_times_restriction_transposed():
    nf = (9, 17)
    nc = tuple(dmg2d._coarse(n) for n in nf)
    R = np.zeros((np.prod(nc), np.prod(nf)))
    for c in range(np.prod(nf)):
        e = np.zeros(nf)
        e.reshape(-1)[c] = 1.0
        R[:, c] = dmg2d.restrict(e).reshape(-1)
    P = np.zeros((np.prod(nf), np.prod(nc)))
    for c in range(np.prod(nc)):
        e = np.zeros(nc)
        e.reshape(-1)[c] = 1.0
        uf = np.zeros(nf)
        dmg2d.prolong_add(e, uf)
        P[:, c] = uf.reshape(-1)
    fi = np.pad(np.ones(tuple(n - 2 for n in nf), dtype=bool), 1).reshape(-1)
    ci = np.pad(np.ones(tuple(n - 2 for n in nc), dtype=bool), 1).reshape(-1)
    # on interior unknowns (the fields are zero on the boundary)
    assert np.abs(P[np.ix_(fi, ci)] - 4.0 * R[np.ix_(ci, fi)].T).max() <= 1e-15


@pytest.mark.parametrize("kw", [dict(), dict(nu1=1, nu2=3, symmetric=True), dict(harmonic=True)])
def test_transposed_cycle_is_the_exact_transpose(kw):
    w = inputs.tissue2d(seed=83, shape=(9, 17))
    H = dmg2d.Hierarchy(w["D"], w["mu"], w["h"], **kw)
    idx = dmg2d.interior_index(w["shape"])
    m = 3
    S = np.zeros((idx.size, idx.size))
    ST = np.zeros_like(S)
    for c in range(idx.size):
        e = np.zeros(w["shape"])
        e.reshape(-1)[idx[c]] = 1.0
        S[:, c] = H.solve(e, fixed=m)[0].reshape(-1)[idx]
        ST[:, c] = H.adjoint(e, fixed=m)[0].reshape(-1)[idx]
    assert np.abs(ST - S.T).max() <= 1e-13 * np.abs(S).max()


def test_first_half_sweep_updates_the_red_vertices():
    # red = even i + j (Sec. 2.2): from u = 0, the colour-0 half-sweep changes
    # exactly the interior vertices with i + j even, the colour-1 one the others
    w = inputs.tissue2d(seed=85, shape=(9, 12))
    ny, nx = w["shape"]
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    inner = (ii > 0) & (jj > 0) & (ii < nx - 1) & (jj < ny - 1)
    f = np.abs(w["q"]) + 1.0
    for colour in (0, 1):
        u = np.zeros(w["shape"])
        dmg2d.gs_half(w["D"], w["mu"], w["h"], f, u, colour)
        assert np.array_equal(u != 0.0, inner & ((ii + jj) % 2 == colour))


@pytest.mark.parametrize("harmonic", [False, True])
def test_gradients_and_tangent_match_finite_differences(harmonic):
    w = inputs.tissue2d(seed=84, shape=(17, 17))
    D, mu, q, h = w["D"], w["mu"], w["q"], w["h"]
    rng = np.random.default_rng(2)
    wv = dmg2d._zero_boundary(rng.standard_normal(D.shape))
    H = dmg2d.Hierarchy(D, mu, h, harmonic=harmonic)
    u, _ = H.solve(q, rtol=1e-13)
    qb, Db, mb, _ = H.vjp(u, wv, rtol=1e-13)
    eps = 1e-6
    inner = dmg2d._zero_boundary(np.ones(D.shape))
    for _ in range(3):
        dq = rng.standard_normal(D.shape)
        dD = 0.1 * D * rng.standard_normal(D.shape)
        dm = 0.1 * mu * rng.standard_normal(D.shape)
        up = dmg2d.direct_solve(D + eps * dD, mu + eps * dm, h, q + eps * dq, harmonic)
        um = dmg2d.direct_solve(D - eps * dD, mu - eps * dm, h, q - eps * dq, harmonic)
        fd = (up - um) / (2 * eps)
        du, _ = H.jvp(u, dq, dD, dm, rtol=1e-13)
        assert np.linalg.norm(du - fd) <= 1e-7 * np.linalg.norm(fd)
        lhs = float(np.sum(wv * fd))
        rhs = float(np.sum(qb * dq * inner) + np.sum(Db * dD) + np.sum(mb * dm))
        assert lhs == pytest.approx(rhs, rel=1e-7)
