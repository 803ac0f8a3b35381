"""dmg_residual_static: the residual norm for callers that may not allocate
device memory (a host framework that owns the whole device pool, or a loop that
cannot take cudaMalloc's implicit synchronisation). It runs from the caller's
arrays and a fixed file-scope scratch array, with no context.

Checked through the C ABI on two calls in a row (the second call must not see
the first call's scratch contents), against the context-based dmg_residual and
against the FP64 CPU oracle's residual, on a small grid and on a thin grid near
the fixed scratch's row limit. This file is collected last so that a run
stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2608_00760_b300 import inputs

torch = pytest.importorskip("torch")

TOL_SAME = 1e-11   # same arithmetic, different rounding order
TOL_ORACLE = 1e-12


def oracle_norms(w, q, u, face_mean):
    """||q - A u|| and ||q|| over interior vertices from the oracle's FP64 residual."""
    m = inputs.interior_mask(w["shape"])
    r = oracle.residual(w["D"], w["mu"], w["h"], q * m, u, harmonic=bool(face_mean))
    return float(np.linalg.norm(r[m])), float(np.linalg.norm(q[m]))


@pytest.fixture(scope="module")
def dmg():
    from paper_2608_00760_b300 import build, dmg
    build.build()
    dmg.lib()
    return dmg


def test_rejects_grids_beyond_the_fixed_scratch(dmg):
    # (ny-2)*(nz-2) = 598^2 rows > 2^18: rejected before any device work
    p = dmg.dmg_default_params(nx=3, ny=600, nz=600, h=1.0)
    st, _ = dmg.dmg_residual_static(p, 1, 1, 1, 1)
    assert st == dmg.DMG_EINVAL
    assert "interior rows" in dmg.dmg_last_error(None)


@pytest.mark.gpu
@pytest.mark.parametrize("face_mean", [0, 1])
def test_matches_context_residual_on_two_calls(dmg, face_mean):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = inputs.tissue(shape=(33, 17, 65), seed=11)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    D, mu = T(w["D"]), T(w["mu"])
    S = dmg.Solver(D, mu, w["h"], face_mean=face_mean, fixed_cycles=2)
    rng = np.random.default_rng(5)
    cases = [(T(w["q"]), T(rng.standard_normal(w["shape"]))),      # r of the size of A u
             (T(w["w"]), None)]                                     # r after two V-cycles
    p = dmg.dmg_default_params(nx=w["shape"][2], ny=w["shape"][1], nz=w["shape"][0], h=w["h"],
                               face_mean=face_mean)
    prev = None
    for q, u in cases:
        if u is None:
            u = S.solve(q)
        ref = S.residual(q, u)
        st, got = dmg.dmg_residual_static(p, D, mu, q, u)
        assert st == dmg.DMG_OK, dmg.dmg_last_error(None)
        assert got[0] == pytest.approx(ref[0], rel=TOL_SAME)
        assert got[1] == pytest.approx(ref[1], rel=TOL_SAME)
        orc = oracle_norms(w, q.cpu().numpy(), u.cpu().numpy(), face_mean)
        assert got[0] == pytest.approx(orc[0], rel=TOL_ORACLE)
        assert got[1] == pytest.approx(orc[1], rel=TOL_ORACLE)
        assert got != prev
        prev = got
    S.close()


@pytest.mark.gpu
def test_near_the_row_limit_matches_the_oracle(dmg):
    # 3 x 513 x 513 vertices: 511^2 = 261,121 interior rows of the 262,144 the
    # scratch holds (about 6 MB per array); two calls with different u
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    shape = (513, 513, 3)
    rng = np.random.default_rng(21)
    w = dict(shape=shape, h=0.5, D=np.exp(0.3 * rng.standard_normal(shape)), mu=np.full(shape, 0.01))
    q = rng.uniform(size=shape)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    p = dmg.dmg_default_params(nx=3, ny=513, nz=513, h=0.5)
    prev = None
    for scale in (0.0, 1.0):
        u = scale * rng.standard_normal(shape)
        st, got = dmg.dmg_residual_static(p, T(w["D"]), T(w["mu"]), T(q), T(u))
        assert st == dmg.DMG_OK, dmg.dmg_last_error(None)
        orc = oracle_norms(w, q, u, 0)
        assert got[0] == pytest.approx(orc[0], rel=TOL_ORACLE)
        assert got[1] == pytest.approx(orc[1], rel=TOL_ORACLE)
        assert got != prev
        prev = got
