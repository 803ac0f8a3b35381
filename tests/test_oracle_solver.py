"""Pins of the oracle's multigrid solver S (Secs. 2.2, Eq. 5).

At convergence S(q) = A^{-1} q, so the V-cycle iteration is checked against a
library sparse direct solve of the oracle's own (separately pinned) operator,
against the closed-form solution for a sine-mode source with constant
coefficients, and for an h-independent contraction factor.
"""
import numpy as np
import pytest

import oracle
from paper_2608_00760_b300 import inputs


@pytest.mark.parametrize("shape", [(9, 9, 9), (17, 17, 17), (17, 9, 33), (5, 5, 9)])
@pytest.mark.parametrize("harmonic", [False, True])
def test_converges_to_direct_solve(shape, harmonic):
    w = inputs.unit_cube(shape=shape, seed=5)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"], harmonic=harmonic)
    u, c, hist = H.solve(w["q"], rtol=1e-12)
    assert hist[-1] <= 1e-12 and c < 30
    ud = oracle.direct_solve(w["D"], w["mu"], w["h"], w["q"], harmonic)
    assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)


def test_tissue_converges_to_direct_solve():
    w = inputs.tissue(17, seed=2)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    u, c, hist = H.solve(w["q"], rtol=1e-12)
    ud = oracle.direct_solve(w["D"], w["mu"], w["h"], w["q"])
    assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)


def test_injection_and_schedule_variants_converge():
    w = inputs.unit_cube(17, seed=4)
    ud = oracle.direct_solve(w["D"], w["mu"], w["h"], w["q"])
    for kw in (dict(inject=True), dict(nu1=1, nu2=1), dict(nu1=3, nu2=0), dict(symmetric=True)):
        H = oracle.Hierarchy(w["D"], w["mu"], w["h"], **kw)
        u, c, hist = H.solve(w["q"], rtol=1e-12, max_cycles=200)
        assert hist[-1] <= 1e-12, kw
        assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud), kw


@pytest.mark.parametrize("p", [(1, 1, 1), (2, 3, 1)])
def test_sine_source_closed_form(p):
    shape, h, Dv, muv = (17, 17, 17), 1.0 / 16, 0.8, 0.5
    c = inputs.constant(shape, h, Dv, muv)
    s = inputs.sine_mode(shape, p)
    lam = Dv / h ** 2 * sum(4 * np.sin(pd * np.pi * h / 2) ** 2 for pd in p) + muv
    H = oracle.Hierarchy(c["D"], c["mu"], h)
    u, _, _ = H.solve(s, rtol=1e-13)
    assert np.abs(u - s / lam).max() <= 1e-11 * np.abs(s / lam).max()


def test_contraction_is_h_independent():
    rates = []
    for n in (17, 33, 65):
        w = inputs.unit_cube(n, seed=0)
        H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
        _, c, hist = H.solve(w["q"], rtol=1e-11)
        rates.append((hist[-1] / hist[2]) ** (1.0 / (len(hist) - 3)))
    assert max(rates) < 0.2 and max(rates) - min(rates) < 0.06, rates


def test_single_level_grid_exact_in_one_cycle():
    rng = np.random.default_rng(0)
    D = np.exp(rng.standard_normal((3, 5, 5)))
    mu = np.full((3, 5, 5), 0.2)
    q = rng.uniform(size=(3, 5, 5))
    H = oracle.Hierarchy(D, mu, 0.1)
    assert H.nlev == 1
    u, c, hist = H.solve(q, rtol=1e-14)
    assert c == 1 and hist[0] < 1e-14
    assert np.allclose(u, oracle.direct_solve(D, mu, 0.1, q), rtol=1e-13, atol=0)


def test_zero_source_and_fixed_cycles():
    w = inputs.unit_cube(9)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    u, c, _ = H.solve(np.zeros(w["shape"]))
    assert c == 0 and not u.any()
    u, c, hist = H.solve(w["q"], fixed=15)
    assert c == 15 and len(hist) == 15
    # the boundary values of q are ignored (Dirichlet)
    q2 = w["q"].copy()
    q2[0] = 7.0
    q2[:, :, -1] = -3.0
    u2, _, _ = H.solve(q2, fixed=15)
    assert np.array_equal(u, u2)
    assert not u[0].any() and not u[:, :, -1].any()
