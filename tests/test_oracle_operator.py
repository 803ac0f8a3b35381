"""Pins of the oracle's discrete operator A (Eq. 1, 7-point finite differences).

Each check ties A to something outside the oracle: the closed-form eigenpairs
of the constant-coefficient operator, the continuous PDE itself (second-order
consistency on a manufactured solution), exact symmetry, and a hand-computed
3x3x3 example stored under tests/golden/.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2608_00760_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("shape", [(9, 9, 9), (17, 9, 33), (5, 17, 9)])
@pytest.mark.parametrize("harmonic", [False, True])
def test_sine_modes_are_eigenvectors(shape, harmonic):
    # constant D, mu: A s_p = lam_p s_p with lam_p = (D/h^2) sum_d 4 sin^2(p_d pi / (2 (n_d-1))) + mu
    h, Dv, muv = 0.37, 1.7, 0.3
    c = inputs.constant(shape, h, Dv, muv)
    for p in [(1, 1, 1), (2, 1, 3), (shape[0] - 2, 1, 2), (3, shape[1] - 2, shape[2] - 2)]:
        s = inputs.sine_mode(shape, p)
        lam = Dv / h ** 2 * sum(4 * np.sin(pd * np.pi / (2 * (n - 1))) ** 2 for pd, n in zip(p, shape)) + muv
        As = oracle.apply(c["D"], c["mu"], h, s, harmonic)
        assert np.abs(As - lam * s).max() <= 1e-12 * lam * np.abs(s).max()


@pytest.mark.parametrize("harmonic", [False, True])
def test_symmetric(harmonic):
    w = inputs.tissue(17, seed=3)
    rng = np.random.default_rng(0)
    m = inputs.interior_mask(w["shape"])
    u = rng.standard_normal(w["shape"]) * m
    v = rng.standard_normal(w["shape"]) * m
    Au = oracle.apply(w["D"], w["mu"], w["h"], u, harmonic)
    Av = oracle.apply(w["D"], w["mu"], w["h"], v, harmonic)
    a, b = np.sum(v * Au), np.sum(Av * u)
    assert abs(a - b) <= 1e-14 * np.sqrt(np.sum(Au ** 2) * np.sum(v ** 2))


@pytest.mark.parametrize("harmonic", [False, True])
def test_positive_definite(harmonic):
    w = inputs.unit_cube(9, seed=1)
    A, _ = oracle.assemble(w["D"], w["mu"], w["h"], harmonic)
    ev = np.linalg.eigvalsh(A.toarray())
    assert ev.min() > 0


def _manufactured(n):
    # u = sin(pi x) sin(pi y) sin(pi z) on the unit cube, D = 1 + 0.5 sin(x + 2y + 3z), mu = 0.3
    h = 1.0 / (n - 1)
    g = np.arange(n) * h
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    u = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    arg = x + 2 * y + 3 * z
    D = 1 + 0.5 * np.sin(arg)
    mu = np.full(u.shape, 0.3)
    # -div(D grad u) + mu u = -D lap u - grad D . grad u + mu u
    lap = -3 * np.pi ** 2 * u
    dDx, dDy, dDz = 0.5 * np.cos(arg), 1.0 * np.cos(arg), 1.5 * np.cos(arg)
    ux = np.pi * np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    uy = np.pi * np.sin(np.pi * x) * np.cos(np.pi * y) * np.sin(np.pi * z)
    uz = np.pi * np.sin(np.pi * x) * np.sin(np.pi * y) * np.cos(np.pi * z)
    Lu = -D * lap - (dDx * ux + dDy * uy + dDz * uz) + mu * u
    return h, D, mu, u, Lu


@pytest.mark.parametrize("harmonic", [False, True])
def test_second_order_consistency_with_pde(harmonic):
    # the discrete A u must approach the continuous operator of Eq. 1 at O(h^2)
    errs = []
    for n in (9, 17, 33):
        h, D, mu, u, Lu = _manufactured(n)
        Au = oracle.apply(D, mu, h, u, harmonic)
        m = inputs.interior_mask(u.shape)
        errs.append(np.abs(Au - Lu)[m].max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.7 < r2 < 4.3, errs


def test_hand_computed_3cube():
    with open(os.path.join(GOLDEN, "hand_3cube.json")) as fh:
        g = json.load(fh)
    D = np.array(g["D"], dtype=float).reshape(3, 3, 3)
    mu = np.array(g["mu"], dtype=float).reshape(3, 3, 3)
    u = np.zeros((3, 3, 3))
    u[1, 1, 1] = g["u_center"]
    for harmonic, key in ((False, "Au_center_arithmetic"), (True, "Au_center_harmonic")):
        Au = oracle.apply(D, mu, g["h"], u, harmonic)
        assert Au[1, 1, 1] == pytest.approx(g[key], rel=1e-15)
        assert np.count_nonzero(Au) == 1
    # the single-unknown solve is exact in one cycle
    H = oracle.Hierarchy(D, mu, g["h"])
    q = np.zeros((3, 3, 3))
    q[1, 1, 1] = g["q_center"]
    x, c, _ = H.solve(q, rtol=1e-14)
    assert c == 1 and x[1, 1, 1] == pytest.approx(g["u_solution_arithmetic"], rel=1e-15)


def test_gauss_seidel_half_sweeps_red_first():
    # Eq. 9 with constant coefficients from u = 0: the red (even i+j+k) half-sweep
    # sets u_p = f_p / diag with diag = 6 D / h^2 + mu; the black half-sweep then
    # uses the updated red neighbours: u_b = (f_b + (D/h^2) sum_red u) / diag.
    shape, h, Dv, muv = (7, 7, 7), 0.25, 1.3, 0.2
    c = inputs.constant(shape, h, Dv, muv)
    rng = np.random.default_rng(0)
    f = rng.uniform(0.5, 1.5, size=shape)
    diag = 6 * Dv / h ** 2 + muv
    u1 = oracle.gs_half(c["D"], c["mu"], h, f, np.zeros(shape), color=0)
    k, j, i = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    red = ((i + j + k) % 2 == 0) & inputs.interior_mask(shape)
    assert np.allclose(u1[red], f[red] / diag, rtol=1e-15)
    assert not u1[~red].any()
    u2 = oracle.gs_half(c["D"], c["mu"], h, f, u1, color=1)
    p = (2, 3, 4)  # black interior point: 2+3+4 odd
    nb = sum(u1[p[0] + a, p[1] + b, p[2] + e] for a, b, e in
             ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)))
    assert u2[p] == pytest.approx((f[p] + Dv / h ** 2 * nb) / diag, rel=1e-14)
    assert np.array_equal(u2[red], u1[red])
