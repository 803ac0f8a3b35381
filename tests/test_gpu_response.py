"""The application's forward model L_e = M(mu S(q)) (Sec. 2.5.3, Eq. response)
through the C ABI: value, tangent and pull-back against the oracle's response
operator, batched samples bitwise equal to single ones, and the autograd
Function against the C ABI."""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("edge", [0.2, 1.0])
@pytest.mark.parametrize("precision", [0, 1])
def test_response_matches_oracle(dmg, edge, precision):
    w = inputs.tissue(33, seed=43)
    rng = np.random.default_rng(5)
    rbar = rng.standard_normal(w["shape"])
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision)
    Le, u = S.response(T(w["q"]), edge)
    dLe = S.response_jvp(u, edge, dq=T(w["dq"]), dD=T(w["dD"]), dmu=T(w["dmu"]))
    qb, Db, mb = S.response_vjp(u, T(rbar), edge)
    S.close()
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    Le_r, u_r = oracle.response(H, w["q"], edge)
    dLe_r = oracle.response_jvp(H, u_r, w["dq"], w["dD"], w["dmu"], edge)
    qb_r, Db_r, mb_r = oracle.response_vjp(H, u_r, rbar, edge)
    assert rel(Le, Le_r) <= 1e-8 and rel(dLe, dLe_r) <= 1e-8
    assert rel(qb, qb_r) <= 1e-8 and rel(Db, Db_r) <= 1e-8 and rel(mb, mb_r) <= 1e-8
    # the masked voxels are exactly zero
    keep = torch.from_numpy(oracle.edge_mask(w["shape"], w["h"], edge)).cuda()
    assert not Le[~keep].any() and not dLe[~keep].any()


def test_response_batch_is_bitwise_single(dmg):
    w = inputs.vi_batch(17, 3, seed=44)
    rbar = np.random.default_rng(6).standard_normal(w["shape"])
    Sb = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    Le, u = Sb.response(T(w["q"]), 1.0)
    qb, Db, mb = Sb.response_vjp(u, T(rbar), 1.0)
    for b in range(3):
        S = dmg.Solver(T(w["D"][b]), T(w["mu"][b]), w["h"])
        Le1, u1 = S.response(T(w["q"][b]), 1.0)
        q1, D1, m1 = S.response_vjp(u1, T(rbar[b]), 1.0)
        assert torch.equal(Le[b], Le1) and torch.equal(u[b], u1)
        assert torch.equal(qb[b], q1) and torch.equal(Db[b], D1) and torch.equal(mb[b], m1)
        S.close()


def test_response_autograd_function(dmg):
    import torch.autograd.forward_ad as fwAD
    from paper_2608_00760_b300 import autograd
    w = inputs.tissue(17, seed=45)
    rbar = T(np.random.default_rng(7).standard_normal(w["shape"]))
    q, D, mu = (T(w[k]).requires_grad_(True) for k in ("q", "D", "mu"))
    Le = autograd.response(q, D, mu, w["h"], 1.0)
    (Le * rbar).sum().backward()
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    Le1, u1 = S.response(T(w["q"]), 1.0)
    qb, Db, mb = S.response_vjp(u1, rbar, 1.0)
    assert torch.equal(Le.detach(), Le1)
    assert torch.equal(q.grad, qb) and torch.equal(D.grad, Db) and torch.equal(mu.grad, mb)
    with fwAD.dual_level():
        out = autograd.response(fwAD.make_dual(T(w["q"]), T(w["dq"])), fwAD.make_dual(T(w["D"]), T(w["dD"])),
                                fwAD.make_dual(T(w["mu"]), T(w["dmu"])), w["h"], 1.0)
        t = fwAD.unpack_dual(out).tangent
    ref = S.response_jvp(u1, 1.0, dq=T(w["dq"]), dD=T(w["dD"]), dmu=T(w["dmu"]))
    assert torch.equal(t, ref)
    # <rbar, J t> = <J^T rbar, t>
    inner = T(inputs.interior_mask(w["shape"]).astype(float))
    lhs = float((rbar * t).sum())
    rhs = float((qb * T(w["dq"]) * inner).sum() + (Db * T(w["dD"])).sum() + (mb * T(w["dmu"])).sum())
    assert lhs == pytest.approx(rhs, rel=1e-8)
    S.close()
    autograd.clear_cache()
