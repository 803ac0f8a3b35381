"""dmg_solve_vjp (forward solve and converged pull-back in one call, host
transfers overlapped on a second stream) gives bit for bit the results of
dmg_solve followed by dmg_vjp, with host or device arrays, FP64 or mixed,
single problems, batches and 2D grids."""
import numpy as np
import pytest

from paper_2608_00760_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_00760_b300 import build, dmg as m
    build.build()
    return m


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


CASES = [
    ("tissue33", lambda: inputs.tissue(33, seed=111), 3),
    ("batch", lambda: inputs.vi_batch(17, 3, seed=112), 3),
    ("2d", lambda: inputs.tissue2d(seed=113, shape=(65, 129)), 2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("host", [False, True])
def test_solve_vjp_is_bitwise_solve_then_vjp(dmg, case, precision, host):
    _, make, dim = case
    w = make()
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision, dim=dim)
    q, wv = T(w["q"]), T(w["w"])
    u = S.solve(q)
    ref = (u,) + S.vjp(u, wv)
    if host:
        qh, wh = (np.ascontiguousarray(w[k]) for k in ("q", "w"))
        outs = [np.zeros(q.shape) for _ in range(4)]
        st = dmg.dmg_solve_vjp(S.ctx, qh, wh, *outs, n=S.n)
        got = [torch.from_numpy(o).cuda() for o in outs]
    else:
        got = [torch.empty_like(q) for _ in range(4)]
        fi, ai = dmg.dmg_info(), dmg.dmg_info()
        st = dmg.dmg_solve_vjp(S.ctx, q, wv, *got, fi, ai, n=S.n)
        assert fi.rel_residual <= 1e-10 and ai.rel_residual <= 1e-10
    assert st == dmg.DMG_OK
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    S.close()
