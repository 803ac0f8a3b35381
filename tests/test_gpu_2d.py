"""The 2D solver (nz = 1: a (ny, nx) grid, 5-point operator) through the C ABI
against the 2D oracle (oracle/dmg2d.py): fixed-cycle schedules and
count-matched adjoints to rounding, converged forward, JVP and VJP to 1e-8 in
FP64 and mixed precision, batches bitwise equal to single problems, a large
grid mixed against FP64, and the 3D-only calls refused."""
import numpy as np
import pytest

from oracle import dmg2d
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


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SHAPES = [(33, 33), (65, 129), (17, 257), (129, 97)]


@pytest.mark.parametrize("shape", SHAPES)
def test_fixed_cycles_and_count_matched_adjoint(dmg, shape):
    w = inputs.tissue2d(seed=91, shape=shape)
    H = dmg2d.Hierarchy(w["D"], w["mu"], w["h"])
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], dim=2, fixed_cycles=4)
    u = S.solve(T(w["q"]))
    ur, _ = H.solve(w["q"], fixed=4)
    assert rel(u, ur) <= 1e-11
    qb, _, _ = S.vjp(u, T(w["w"]), cycles=4, need=(True, False, False))
    lr, _ = H.adjoint(w["w"], fixed=4)
    assert rel(qb, lr) <= 1e-11
    S.close()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", [0, 1])
def test_converged_forward_jvp_vjp(dmg, shape, precision):
    w = inputs.tissue2d(seed=92, shape=shape)
    H = dmg2d.Hierarchy(w["D"], w["mu"], w["h"])
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], dim=2, precision=precision)
    u = S.solve(T(w["q"]))
    assert S.last_info.rel_residual <= 1e-10
    du = S.jvp(u, T(w["dq"]), T(w["dD"]), T(w["dmu"]))
    qb, Db, mb = S.vjp(u, T(w["w"]))
    S.close()
    ur, _ = H.solve(w["q"], rtol=1e-10)
    dur, _ = H.jvp(ur, w["dq"], w["dD"], w["dmu"], rtol=1e-10)
    qr, Dr, mr, _ = H.vjp(ur, w["w"], rtol=1e-10)
    for got, ref in ((u, ur), (du, dur), (qb, qr), (Db, Dr), (mb, mr)):
        assert rel(got, ref) <= 1e-8


def test_2d_batch_is_bitwise_single(dmg):
    ws = [inputs.tissue2d(seed=(93, b), shape=(33, 65)) for b in range(3)]
    st = lambda k: np.stack([x[k] for x in ws])
    Sb = dmg.Solver(T(st("D")), T(st("mu")), 0.5, dim=2, precision=1)
    ub = Sb.solve(T(st("q")))
    qb, Db, mb = Sb.vjp(ub, T(st("w")))
    Sb.close()
    for b in range(3):
        S = dmg.Solver(T(ws[b]["D"]), T(ws[b]["mu"]), 0.5, dim=2, precision=1)
        u = S.solve(T(ws[b]["q"]))
        q1, D1, m1 = S.vjp(u, T(ws[b]["w"]))
        S.close()
        assert torch.equal(ub[b], u)
        assert torch.equal(qb[b], q1) and torch.equal(Db[b], D1) and torch.equal(mb[b], m1)


def test_large_2d_mixed_matches_fp64(dmg):
    n = 4097
    g = torch.Generator(device="cuda").manual_seed(5)
    D = 0.3 * torch.exp(0.3 * torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64))
    mu = torch.full((n, n), 0.01, device="cuda", dtype=torch.float64)
    q = torch.rand((n, n), generator=g, device="cuda", dtype=torch.float64)
    out = {}
    for prec in (0, 1):
        S = dmg.Solver(D, mu, 0.5, dim=2, precision=prec)
        u = S.solve(q)
        assert S.last_info.rel_residual <= 1e-10
        out[prec] = u
        S.close()
    assert float(torch.linalg.norm(out[1] - out[0]) / torch.linalg.norm(out[0])) <= 1e-8


def test_3d_only_calls_are_refused(dmg):
    w = inputs.tissue2d(seed=94, shape=(17, 17))
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], dim=2)
    x = T(w["q"])
    assert dmg.dmg_vjp_unrolled(S.ctx, x, x, 2, 0, None, None, None, None, n=S.n) == dmg.DMG_EINVAL
    assert dmg.dmg_response(S.ctx, x, 1.0, torch.empty_like(x), n=S.n) == dmg.DMG_EINVAL
    S.close()
