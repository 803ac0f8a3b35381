"""Pins of the oracle's response operator R(q) = M(mu S(q)) (Sec. 2.5.3,
Eq. response): the edge mask against a hand count, R against a library direct
solve, and its JVP / VJP against central finite differences of R built from
direct solves (so the explicit factor mu and the masked cotangent are both
exercised)."""
import numpy as np
import pytest

import oracle
from paper_2608_00760_b300 import inputs


def test_edge_mask_counts():
    # h = 0.5: edge 0.2 keeps indices 1..n-2 (0.5 >= 0.2), edge 1.0 keeps 2..n-3,
    # edge 0.5 keeps 1..n-2 (exactly one spacing), edge 0 keeps everything
    shape = (9, 11, 13)
    assert oracle.edge_mask(shape, 0.5, 0.0).sum() == 9 * 11 * 13
    assert oracle.edge_mask(shape, 0.5, 0.2).sum() == 7 * 9 * 11
    assert oracle.edge_mask(shape, 0.5, 0.5).sum() == 7 * 9 * 11
    assert oracle.edge_mask(shape, 0.5, 1.0).sum() == 5 * 7 * 9
    assert oracle.edge_mask(shape, 0.5, 1.01).sum() == 3 * 5 * 7
    m = oracle.edge_mask(shape, 0.5, 1.0)
    assert m[2, 2, 2] and m[-3, -3, -3] and not m[1, 5, 5] and not m[4, -2, 5]


def test_response_matches_direct_solve():
    w = inputs.tissue(9, seed=41)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    Le, u = oracle.response(H, w["q"], 1.0, rtol=1e-13)
    ud = oracle.direct_solve(w["D"], w["mu"], w["h"], w["q"])
    ref = np.where(oracle.edge_mask(w["shape"], w["h"], 1.0), w["mu"] * ud, 0.0)
    assert np.linalg.norm(Le - ref) <= 1e-11 * np.linalg.norm(ref)


def _R_direct(D, mu, h, q, edge):
    u = oracle.direct_solve(D, mu, h, q)
    return np.where(oracle.edge_mask(D.shape, h, edge), mu * u, 0.0)


@pytest.mark.parametrize("edge", [0.2, 1.0])
def test_response_derivatives_match_finite_differences(edge):
    w = inputs.tissue(9, seed=42)
    D, mu, q, h = w["D"], w["mu"], w["q"], w["h"]
    rng = np.random.default_rng(4)
    rbar = rng.standard_normal(D.shape)
    H = oracle.Hierarchy(D, mu, h)
    Le, u = oracle.response(H, q, edge, rtol=1e-13)
    qb, Db, mb = oracle.response_vjp(H, u, rbar, edge, rtol=1e-13)
    eps = 1e-6
    for _ in range(3):
        dq = rng.standard_normal(D.shape)
        dD = 0.1 * D * rng.standard_normal(D.shape)
        dm = 0.1 * mu * rng.standard_normal(D.shape)
        fd = (_R_direct(D + eps * dD, mu + eps * dm, h, q + eps * dq, edge) -
              _R_direct(D - eps * dD, mu - eps * dm, h, q - eps * dq, edge)) / (2 * eps)
        jv = oracle.response_jvp(H, u, dq, dD, dm, edge, rtol=1e-13)
        assert np.linalg.norm(jv - fd) <= 1e-7 * np.linalg.norm(fd)
        lhs = float(np.sum(rbar * fd))
        # q on boundary vertices is ignored (Dirichlet): its cotangent entries there do not enter
        inner = inputs.interior_mask(D.shape)
        rhs = float(np.sum(qb * dq * inner) + np.sum(Db * dD) + np.sum(mb * dm))
        assert lhs == pytest.approx(rhs, rel=1e-7)
