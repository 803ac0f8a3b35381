"""torch.autograd.Function around the C ABI: reverse mode (the hand-written
adjoint V-cycle + gradient kernel) and forward mode (dmg_jvp), checked against
the FP64 oracle's gradients and against central finite differences of the
solve itself."""
import numpy as np
import pytest

import oracle
from paper_2608_00760_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_00760_b300 import autograd, build
    build.build()
    return autograd


def T(a, grad=False):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda", requires_grad=grad)


@pytest.mark.parametrize("recompute", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_backward_matches_oracle(ag, recompute, precision):
    w = inputs.tissue(33, seed=21)
    q, D, mu = T(w["q"], True), T(w["D"], True), T(w["mu"], True)
    u = ag.solve(q, D, mu, w["h"], recompute=recompute, precision=precision)
    (u * T(w["w"])).sum().backward()
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ur, _, _ = H.solve(w["q"], rtol=1e-10)
    qbr, Dbr, mbr, _ = H.vjp(ur, w["w"], rtol=1e-10)
    for got, ref in ((q.grad, qbr), (D.grad, Dbr), (mu.grad, mbr)):
        g = got.cpu().numpy()
        assert np.linalg.norm(g - ref) <= 1e-8 * np.linalg.norm(ref)


def test_gradients_match_finite_differences(ag):
    # central differences of <w, u> through the solve at rtol 1e-13 (step 1e-6)
    w = inputs.tissue(17, seed=22)
    rng = np.random.default_rng(3)
    q, D, mu = T(w["q"], True), T(w["D"], True), T(w["mu"], True)
    W = T(w["w"])
    loss = lambda qq, DD, mm: float((ag.solve(qq, DD, mm, w["h"], rtol=1e-13) * W).sum())
    u = ag.solve(q, D, mu, w["h"], rtol=1e-13)
    (u * W).sum().backward()
    eps = 1e-6
    for _ in range(5):
        dq = T(rng.standard_normal(w["shape"]))
        dD = T(rng.standard_normal(w["shape"]) * w["D"])
        dm = T(rng.standard_normal(w["shape"]) * w["mu"])
        with torch.no_grad():
            fd = (loss(q + eps * dq, D + eps * dD, mu + eps * dm) -
                  loss(q - eps * dq, D - eps * dD, mu - eps * dm)) / (2 * eps)
        an = float((q.grad * dq).sum() + (D.grad * dD).sum() + (mu.grad * dm).sum())
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(an))


@pytest.mark.parametrize("recompute", [False, True])
def test_forward_mode_matches_jvp_and_duality(ag, recompute):
    import torch.autograd.forward_ad as fwAD
    w = inputs.tissue(17, seed=23)
    q, D, mu = T(w["q"]), T(w["D"]), T(w["mu"])
    dq, dD, dm = T(w["dq"]), T(w["dD"]), T(w["dmu"])
    with fwAD.dual_level():
        out = ag.solve(fwAD.make_dual(q, dq), fwAD.make_dual(D, dD), fwAD.make_dual(mu, dm), w["h"],
                       recompute=recompute)
        du = fwAD.unpack_dual(out).tangent
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ur, _, _ = H.solve(w["q"], rtol=1e-10)
    ref, _ = H.jvp(ur, w["dq"], w["dD"], w["dmu"], rtol=1e-10)
    assert np.linalg.norm(du.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    # <w, J t> = <J^T w, t>
    qg, Dg, mg = T(w["q"], True), T(w["D"], True), T(w["mu"], True)
    (ag.solve(qg, Dg, mg, w["h"]) * T(w["w"])).sum().backward()
    lhs = float((du * T(w["w"])).sum())
    m = T(inputs.interior_mask(w["shape"]).astype(float))
    rhs = float((qg.grad * dq * m).sum() + (Dg.grad * dD).sum() + (mg.grad * dm).sum())
    assert lhs == pytest.approx(rhs, rel=1e-8)


def test_cache_tracks_coefficient_changes(ag):
    w = inputs.unit_cube(17, seed=24)
    q, D, mu = T(w["q"]), T(w["D"]), T(w["mu"])
    u1 = ag.solve(q, D, mu, w["h"])
    with torch.no_grad():
        D.mul_(2.0)          # in-place change bumps the version: a new context is built
    u2 = ag.solve(q, D, mu, w["h"])
    H = oracle.Hierarchy(2.0 * w["D"], w["mu"], w["h"])
    ref, _, _ = H.solve(w["q"], rtol=1e-10)
    assert np.linalg.norm(u2.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    assert not torch.allclose(u1, u2)
