"""The unrolled coefficient gradient (dmg_vjp_unrolled): the exact derivative of
<w, S_m(q; D, mu)> for m FP64 V-cycles, through every iterate and the coarsened
coefficients, against the complex-step oracle (oracle/unrolled.py) entry by
entry and along random directions, with the iterate and qbar against the C
oracle's fixed-cycle solve and count-matched adjoint."""
import numpy as np
import pytest

import oracle
from oracle import unrolled
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


def N(t):
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_gradient_entries_match_complex_step(dmg):
    w = inputs.tissue(seed=61, shape=(5, 9, 9))
    wv = np.random.default_rng(11).standard_normal(w["shape"])
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    u, qb, Db, mb = S.vjp_unrolled(T(w["q"]), T(wv), 2)
    S.close()
    qr, Dr, mr = unrolled.gradient(w["D"], w["mu"], w["h"], w["q"], wv, 2)
    inner = inputs.interior_mask(w["shape"])
    assert np.abs(N(qb) - qr * inner).max() <= 1e-10 * np.abs(qr).max()
    assert np.abs(N(Db) - Dr).max() <= 1e-10 * np.abs(Dr).max()
    assert np.abs(N(mb) - mr).max() <= 1e-10 * np.abs(mr).max()


CASES = [
    dict(shape=(17, 17, 17), m=1, kw={}),
    dict(shape=(17, 17, 17), m=5, kw={}),
    dict(shape=(9, 17, 33), m=3, kw={}),
    dict(shape=(17, 17, 17), m=3, kw=dict(nu1=1, nu2=3, symmetric=1)),
    dict(shape=(17, 17, 17), m=3, kw=dict(nu1=0, nu2=2)),
    dict(shape=(17, 17, 17), m=3, kw=dict(face_mean=1)),
    dict(shape=(17, 17, 17), m=3, kw=dict(coarsen=1)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-m%d-%s" % ("x".join(map(str, c["shape"])), c["m"], c["kw"]))
def test_directional_derivatives_match_complex_step(dmg, case):
    w = inputs.tissue(seed=62, shape=case["shape"])
    rng = np.random.default_rng(12)
    wv = rng.standard_normal(w["shape"])
    kw, m = case["kw"], case["m"]
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], **kw)
    u, qb, Db, mb = S.vjp_unrolled(T(w["q"]), T(wv), m)
    S.close()
    okw = dict(nu1=kw.get("nu1", 2), nu2=kw.get("nu2", 2), symmetric=bool(kw.get("symmetric", 0)),
               harmonic=bool(kw.get("face_mean", 0)), inject=bool(kw.get("coarsen", 0)))
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"], **okw)
    ur, _, _ = H.solve(w["q"], fixed=m)
    assert rel(N(u), ur) <= 1e-12
    lam, _, _ = H.adjoint(wv, fixed=m)
    assert rel(N(qb), lam) <= 1e-11
    for _ in range(3):
        dD = 0.2 * w["D"] * rng.standard_normal(w["shape"])
        dm = 0.2 * w["mu"] * rng.standard_normal(w["shape"])
        cs = unrolled.directional(w["D"], w["mu"], w["h"], w["q"], wv, m, dD=dD, dmu=dm, **okw)
        an = float(np.sum(N(Db) * dD) + np.sum(N(mb) * dm))
        assert an == pytest.approx(cs, rel=1e-9)


def test_checkpoint_stride_does_not_change_the_result(dmg):
    w = inputs.tissue(seed=63, shape=(17, 17, 33))
    wv = T(np.random.default_rng(13).standard_normal(w["shape"]))
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    ref = S.vjp_unrolled(T(w["q"]), wv, 7, stride=1)
    for stride in (0, 2, 3, 7, 10):
        got = S.vjp_unrolled(T(w["q"]), wv, 7, stride=stride)
        assert all(torch.equal(a, b) for a, b in zip(got, ref)), stride
    S.close()


def test_many_cycles_tend_to_the_converged_gradient(dmg):
    w = inputs.tissue(seed=64, shape=(17, 17, 17))
    wv = T(np.random.default_rng(14).standard_normal(w["shape"]))
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], rtol=1e-13)
    u, qb, Db, mb = S.vjp_unrolled(T(w["q"]), wv, 40)
    uc = S.solve(T(w["q"]))
    qc, Dc, mc = S.vjp(uc, wv)
    S.close()
    for a, b in ((u, uc), (qb, qc), (Db, Dc), (mb, mc)):
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) <= 1e-9


def test_unrolled_batch_is_bitwise_single(dmg):
    w = inputs.vi_batch(17, 3, seed=65)
    wv = np.random.default_rng(15).standard_normal(w["shape"])
    Sb = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    out = Sb.vjp_unrolled(T(w["q"]), T(wv), 4)
    Sb.close()
    for b in range(3):
        S = dmg.Solver(T(w["D"][b]), T(w["mu"][b]), w["h"])
        one = S.vjp_unrolled(T(w["q"][b]), T(wv[b]), 4)
        S.close()
        assert all(torch.equal(x[b], y) for x, y in zip(out, one)), b


def test_autograd_unrolled_backward(dmg):
    from paper_2608_00760_b300 import autograd
    w = inputs.tissue(seed=66, shape=(17, 17, 17))
    wv = T(np.random.default_rng(16).standard_normal(w["shape"]))
    q, D, mu = (T(w[k]).requires_grad_(True) for k in ("q", "D", "mu"))
    u = autograd.solve(q, D, mu, w["h"], unrolled=True, fixed_cycles=6)
    (u * wv).sum().backward()
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], fixed_cycles=6)
    u6 = S.solve(T(w["q"]))
    _, qb, Db, mb = S.vjp_unrolled(T(w["q"]), wv, 6)
    S.close()
    assert torch.equal(u.detach(), u6)
    assert torch.equal(q.grad, qb) and torch.equal(D.grad, Db) and torch.equal(mu.grad, mb)
    autograd.clear_cache()
