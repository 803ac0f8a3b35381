"""Pins of the oracle's adjoint solver S^dagger (Sec. 2.4, Eq. 18).

The fixed-count map S_m (m V-cycles from zero, the paper's matched-count mode)
is linear in q, so its adjoint is its matrix transpose. The oracle computes it
two ways, the literal reversed composition of per-operation adjoints
(Eqs. 10-11, 15-16, 17) and the transposed V-cycle iteration; both are checked
against the explicit transpose of S_m built column by column, and against each
other and the dot-product identity on larger grids.
"""
import numpy as np
import pytest

import oracle
from paper_2608_00760_b300 import inputs


def explicit(fn, shape):
    idx = oracle.interior_index(shape)
    M = np.zeros((idx.size, idx.size))
    e = np.zeros(shape)
    ef = e.reshape(-1)
    for c in range(idx.size):
        ef[idx[c]] = 1.0
        M[:, c] = fn(e).reshape(-1)[idx]
        ef[idx[c]] = 0.0
    return M


@pytest.mark.parametrize("shape,m", [((5, 5, 5), 1), ((5, 5, 5), 3), ((9, 9, 9), 2), ((9, 5, 9), 2)])
@pytest.mark.parametrize("harmonic", [False, True])
def test_brute_force_transpose(shape, m, harmonic):
    w = inputs.unit_cube(shape=shape, seed=7)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"], harmonic=harmonic)
    S = explicit(lambda e: H.solve(e, fixed=m)[0], shape)
    ST = explicit(lambda e: H.adjoint(e, fixed=m)[0], shape)
    SL = explicit(lambda e: H.adjoint_literal(e, m), shape)
    scale = np.abs(S).max()
    assert np.abs(ST - S.T).max() <= 1e-13 * scale
    assert np.abs(SL - S.T).max() <= 1e-13 * scale
    # the forward schedule (red->black pre and post) is not symmetric
    assert np.abs(S - S.T).max() > 1e-6 * scale


@pytest.mark.parametrize("nu1,nu2,symmetric", [(1, 3, False), (3, 1, False), (1, 2, True)])
def test_brute_force_transpose_with_unequal_sweep_counts(nu1, nu2, symmetric):
    # the transposed cycle runs nu2 pre- and nu1 post-sweeps (Sec. 2.4); with
    # nu1 != nu2 a cycle that kept the forward counts would not be the transpose
    shape = (9, 5, 9)
    w = inputs.unit_cube(shape=shape, seed=11)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"], nu1=nu1, nu2=nu2, symmetric=symmetric)
    S = explicit(lambda e: H.solve(e, fixed=2)[0], shape)
    ST = explicit(lambda e: H.adjoint(e, fixed=2)[0], shape)
    SL = explicit(lambda e: H.adjoint_literal(e, 2), shape)
    scale = np.abs(S).max()
    assert np.abs(ST - S.T).max() <= 1e-13 * scale
    assert np.abs(SL - S.T).max() <= 1e-13 * scale


def test_symmetric_schedule_special_case():
    # post-smoothing black->red with nu1 == nu2 makes the V-cycle symmetric: S_m^T = S_m
    w = inputs.unit_cube(shape=(9, 9, 9), seed=8)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"], symmetric=True)
    S = explicit(lambda e: H.solve(e, fixed=2)[0], (9, 9, 9))
    assert np.abs(S - S.T).max() <= 1e-13 * np.abs(S).max()


@pytest.mark.parametrize("n,m", [(17, 4), (33, 3)])
def test_literal_equals_transposed_cycle_and_dot_test(n, m):
    w = inputs.tissue(n, seed=9)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    a = H.adjoint(w["w"], fixed=m)[0]
    b = H.adjoint_literal(w["w"], m)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    msk = inputs.interior_mask(w["shape"])
    v = w["dq"] * msk
    Sv = H.solve(v, fixed=m)[0]
    lhs, rhs = np.sum(w["w"][msk] * Sv[msk]), np.sum(a[msk] * v[msk])
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(w["w"]) * np.linalg.norm(Sv)


def test_converged_adjoint_is_inverse():
    w = inputs.unit_cube(17, seed=10)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    lam, c, hist = H.adjoint(w["w"], rtol=1e-12)
    ref = oracle.direct_solve(w["D"], w["mu"], w["h"], w["w"])
    assert np.linalg.norm(lam - ref) <= 1e-9 * np.linalg.norm(ref)
