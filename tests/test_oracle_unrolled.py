"""Pins of the unrolled-gradient oracle (oracle/unrolled.py): its V-cycle in
real arithmetic reproduces the C oracle's fixed-cycle solve; its complex-step
derivatives agree with central finite differences of the C oracle's
fixed-cycle solve; the entry-by-entry gradient is consistent with directional
derivatives; and for many cycles the unrolled derivative tends to the
derivative of the exact solution (the adjoint-state gradient)."""
import numpy as np
import pytest

import oracle
from oracle import unrolled
from paper_2608_00760_b300 import inputs


@pytest.mark.parametrize("shape", [(17, 17, 17), (9, 17, 33)])
@pytest.mark.parametrize("m", [1, 3])
def test_real_vcycle_matches_c_oracle(shape, m):
    w = inputs.tissue(seed=51, shape=shape)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ref, _, _ = H.solve(w["q"], fixed=m)
    u = unrolled.solve_fixed(w["D"], w["mu"], w["h"], w["q"], m)
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)


def test_complex_step_matches_finite_differences_of_c_oracle():
    w = inputs.tissue(seed=52, shape=(9, 17, 17))
    D, mu, q, h = w["D"], w["mu"], w["q"], w["h"]
    rng = np.random.default_rng(8)
    wv = rng.standard_normal(D.shape)
    m = 3
    eps = 1e-5

    def L(Dp, mp, qp):
        u, _, _ = oracle.Hierarchy(Dp, mp, h).solve(qp, fixed=m)
        return float(np.sum(wv * u))

    for _ in range(3):
        dq = rng.standard_normal(D.shape)
        dD = 0.2 * D * rng.standard_normal(D.shape)
        dm = 0.2 * mu * rng.standard_normal(D.shape)
        fd = (L(D + eps * dD, mu + eps * dm, q + eps * dq) - L(D - eps * dD, mu - eps * dm, q - eps * dq)) / (2 * eps)
        cs = unrolled.directional(D, mu, h, q, wv, m, dq=dq, dD=dD, dmu=dm)
        assert cs == pytest.approx(fd, rel=1e-7)


def test_gradient_entries_are_consistent_with_directions():
    w = inputs.tissue(seed=53, shape=(5, 5, 9))
    rng = np.random.default_rng(9)
    wv = rng.standard_normal(w["shape"])
    qb, Db, mb = unrolled.gradient(w["D"], w["mu"], w["h"], w["q"], wv, 2)
    dq, dD, dm = (rng.standard_normal(w["shape"]) for _ in range(3))
    cs = unrolled.directional(w["D"], w["mu"], w["h"], w["q"], wv, 2, dq=dq, dD=dD, dmu=dm)
    assert float(np.sum(qb * dq) + np.sum(Db * dD) + np.sum(mb * dm)) == pytest.approx(cs, rel=1e-10)
    # q on boundary vertices is ignored: its gradient there is exactly zero
    assert not qb[0].any() and not qb[:, :, -1].any()


def test_many_cycles_tend_to_the_exact_solution_gradient():
    w = inputs.tissue(seed=54, shape=(9, 9, 17))
    D, mu, q, h = w["D"], w["mu"], w["q"], w["h"]
    rng = np.random.default_rng(10)
    wv = rng.standard_normal(D.shape)
    H = oracle.Hierarchy(D, mu, h)
    u, _, _ = H.solve(q, rtol=1e-14, max_cycles=200)
    qb, Db, mb, _ = H.vjp(u, wv, rtol=1e-14, max_cycles=200)
    dD = 0.2 * D * rng.standard_normal(D.shape)
    dm = 0.2 * mu * rng.standard_normal(D.shape)
    cs = unrolled.directional(D, mu, h, q, wv, 40, dD=dD, dmu=dm)
    assert cs == pytest.approx(float(np.sum(Db * dD) + np.sum(mb * dm)), rel=1e-9)
