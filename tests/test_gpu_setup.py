"""Row a1 beyond the first setup: dmg_set_coefficients rebuilds the
coefficient hierarchy of an existing context in place (the per-iteration
setup of a variational-inference loop, whose coefficients change every
iteration). Checked through the C ABI: after new coefficients, solve and
gradients are bit for bit those of a context set up with them from the start
(single and batched, FP64 and mixed), the captured graphs keep working, and a
non-positive-definite field is refused. Also the instrumentation probe of the
FMA rate that the benchmark uses as its FP64 roofline denominator."""
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


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("batch", [1, 3])
def test_new_coefficients_equal_a_fresh_setup(dmg, precision, batch):
    shape = (17, 33, 33)
    a = [inputs.tissue(seed=(40, b), shape=shape) for b in range(batch)]
    b = [inputs.tissue(seed=(41, b), shape=shape) for b in range(batch)]
    st = lambda ws, k: T(np.stack([w[k] for w in ws])) if batch > 1 else T(ws[0][k])
    S = dmg.Solver(st(a, "D"), st(a, "mu"), 0.5, precision=precision)
    u_a = S.solve(st(a, "q"))                   # graphs captured with the first coefficients
    S.set_coefficients(st(b, "D"), st(b, "mu"))
    u = S.solve(st(b, "q"))
    qb, Db, mb = S.vjp(u, st(b, "w"))
    F = dmg.Solver(st(b, "D"), st(b, "mu"), 0.5, precision=precision)
    uf = F.solve(st(b, "q"))
    qf, Df, mf = F.vjp(uf, st(b, "w"))
    for x, y in ((u, uf), (qb, qf), (Db, Df), (mb, mf)):
        assert torch.equal(x, y)
    assert not torch.equal(u, u_a)
    # and against the oracle on the new coefficients
    H = oracle.Hierarchy(b[0]["D"], b[0]["mu"], 0.5)
    ur, _, _ = H.solve(b[0]["q"], rtol=1e-10)
    u0 = (u[0] if batch > 1 else u).cpu().numpy()
    assert np.linalg.norm(u0 - ur) <= 1e-8 * np.linalg.norm(ur)
    S.close()
    F.close()


def test_set_coefficients_refuses_indefinite_fields(dmg):
    w = inputs.tissue(seed=42, shape=(17, 17, 17))
    S = dmg.Solver(T(w["D"]), T(w["mu"]), 0.5)
    st = dmg.dmg_set_coefficients(S.ctx, T(-w["D"]), T(w["mu"]), None, n=S.n)
    assert st == dmg.DMG_EINVAL and "positive definite" in dmg.dmg_last_error(S.ctx)
    assert dmg.dmg_set_coefficients(S.ctx, None, T(w["mu"]), None, n=S.n) == dmg.DMG_EINVAL
    S.set_coefficients(T(w["D"]), T(w["mu"]))   # usable again after good coefficients
    u = S.solve(T(w["q"]))
    assert S.last_info.rel_residual <= 1e-10 and bool(torch.isfinite(u).all())
    S.close()


def test_fma_probe_reports_plausible_rates(dmg):
    st, r64 = dmg.dmg_probe_fma(True)
    assert st == dmg.DMG_OK
    st, r32 = dmg.dmg_probe_fma(False)
    assert st == dmg.DMG_OK
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # at most 2 FP64 and 128 FP32 FMA per clock per SM at up to 2.2 GHz; at least a tenth of that
    assert 0.1 * 2 * sms * 2.2e9 < r64 <= 2 * sms * 2.2e9
    assert 0.1 * 128 * sms * 2.2e9 < r32 <= 128 * sms * 2.2e9
