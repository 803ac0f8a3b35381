"""Pins of the oracle's coefficient derivatives (an extension beyond the paper,
whose Sec. 4 lists differentiation w.r.t. D and the absorption as future work).

For L = <w, u>, A(D, mu) u = q: dL = -lam^T (dA) u with lam = A^{-1} w. The
gradients and the tangent operator are checked against central finite
differences of the library direct solve and of the operator, and against the
closed forms for constant coefficients with sine-mode source and cotangent.
"""
import numpy as np
import pytest

import oracle
from paper_2608_00760_b300 import inputs


def _loss(D, mu, h, q, w, harmonic):
    return np.sum(w * oracle.direct_solve(D, mu, h, q, harmonic))


@pytest.mark.parametrize("harmonic", [False, True])
def test_gradients_match_central_differences(harmonic):
    wl = inputs.tissue(9, seed=11)
    D, mu, h, q = wl["D"], wl["mu"], wl["h"], wl["q"]
    rng = np.random.default_rng(3)
    w = rng.standard_normal(D.shape) * inputs.interior_mask(D.shape)
    u = oracle.direct_solve(D, mu, h, q, harmonic)
    lam = oracle.direct_solve(D, mu, h, w, harmonic)
    Db, mb = oracle.grad(D, h, u, lam, harmonic)
    for _ in range(3):
        dD = rng.standard_normal(D.shape) * D          # every vertex, boundary included
        dmu = rng.standard_normal(D.shape) * mu
        eps = 1e-5
        fd_D = (_loss(D + eps * dD, mu, h, q, w, harmonic) - _loss(D - eps * dD, mu, h, q, w, harmonic)) / (2 * eps)
        fd_m = (_loss(D, mu + eps * dmu, h, q, w, harmonic) - _loss(D, mu - eps * dmu, h, q, w, harmonic)) / (2 * eps)
        assert np.sum(Db * dD) == pytest.approx(fd_D, rel=1e-7)
        assert np.sum(mb * dmu) == pytest.approx(fd_m, rel=1e-7)
    # mu on the boundary has no effect; D on the boundary does
    m = inputs.interior_mask(D.shape)
    assert not mb[~m].any()
    assert np.abs(Db[~m]).max() > 0


def test_constant_coefficient_closed_forms():
    shape, h, Dv, muv = (17, 17, 17), 1.0 / 16, 0.9, 0.4
    c = inputs.constant(shape, h, Dv, muv)
    p = (1, 2, 1)
    s = inputs.sine_mode(shape, p)
    lam_p = Dv / h ** 2 * sum(4 * np.sin(pd * np.pi * h / 2) ** 2 for pd in p) + muv
    u = s / lam_p                   # exact discrete solution for q = s
    lam = s / lam_p                 # adjoint state for w = s
    Db, mb = oracle.grad(c["D"], h, u, lam)
    wq = np.sum(s * s)
    # d/dmu (uniform shift) <w,u> = -<w,q>/lam_p^2
    assert np.sum(mb) == pytest.approx(-wq / lam_p ** 2, rel=1e-12)
    # uniform scaling D(1+eps): d/deps <w,u> = -(lam_p - mu) <w,q> / lam_p^2
    assert np.sum(Db * c["D"]) == pytest.approx(-(lam_p - muv) * wq / lam_p ** 2, rel=1e-12)


@pytest.mark.parametrize("harmonic", [False, True])
def test_tangent_operator_matches_difference_of_operators(harmonic):
    wl = inputs.unit_cube(9, seed=12)
    D, mu, h = wl["D"], wl["mu"], wl["h"]
    rng = np.random.default_rng(4)
    u = rng.standard_normal(D.shape) * inputs.interior_mask(D.shape)
    dD, dmu = wl["dD"], wl["dmu"]
    # A is linear in (D, mu) for the arithmetic mean, so a unit step is exact;
    # the harmonic mean needs a small step (truncation O(eps^2))
    eps = 1.0 if not harmonic else 1e-4
    fd = (oracle.apply(D + eps * dD, mu + eps * dmu, h, u, harmonic)
          - oracle.apply(D - eps * dD, mu - eps * dmu, h, u, harmonic)) / (2 * eps)
    out = oracle.dA_apply(D, h, dD, dmu, u, harmonic)
    tol = 1e-13 if not harmonic else 1e-7
    assert np.abs(out - fd).max() <= tol * np.abs(fd).max()


@pytest.mark.parametrize("harmonic", [False, True])
def test_jvp_vjp_duality_and_fd(harmonic):
    wl = inputs.tissue(9, seed=13)
    D, mu, h, q = wl["D"], wl["mu"], wl["h"], wl["q"]
    H = oracle.Hierarchy(D, mu, h, harmonic=harmonic)
    u, _, _ = H.solve(q, rtol=1e-13)
    du, _ = H.jvp(u, wl["dq"], wl["dD"], wl["dmu"], rtol=1e-13)
    qb, Db, mb, _ = H.vjp(u, wl["w"], rtol=1e-13)
    m = inputs.interior_mask(D.shape)
    lhs = np.sum(wl["w"][m] * du[m])
    rhs = np.sum(qb[m] * wl["dq"][m]) + np.sum(Db * wl["dD"]) + np.sum(mb * wl["dmu"])
    assert lhs == pytest.approx(rhs, rel=1e-10)
    eps = 1e-5
    up = oracle.direct_solve(D + eps * wl["dD"], mu + eps * wl["dmu"], h, q + eps * wl["dq"], harmonic)
    um = oracle.direct_solve(D - eps * wl["dD"], mu - eps * wl["dmu"], h, q - eps * wl["dq"], harmonic)
    fd = (up - um) / (2 * eps)
    assert np.linalg.norm(du - fd) <= 1e-7 * np.linalg.norm(fd)
