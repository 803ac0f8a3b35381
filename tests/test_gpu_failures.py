"""Failure detection without a GPU fault: allocation failures injected on the
host (dmg_debug_fail_alloc) or real ones (a request far above the device
memory) return DMG_ENOMEM, release what was allocated, and leave the process
and other contexts usable; a failed work-buffer allocation of the unrolled
gradient leaves its context usable."""
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


@pytest.mark.parametrize("k", [1, 7, 30, 60])
def test_injected_setup_failure_then_recovery(dmg, k):
    w = inputs.tissue(17, seed=101)
    p = dmg.dmg_default_params(nx=17, ny=17, nz=17, h=w["h"], precision=1)
    free0 = torch.cuda.mem_get_info()[0]
    dmg.dmg_debug_fail_alloc(k)
    try:
        st, ctx = dmg.dmg_setup(p, T(w["D"]), T(w["mu"]))
    finally:
        dmg.dmg_debug_fail_alloc(0)
    assert st == dmg.DMG_ENOMEM and ctx is None and "injected" in dmg.dmg_last_error(None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)   # what was allocated was released
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1)
    S.solve(T(w["q"]))
    assert S.last_info.rel_residual <= 1e-10
    S.close()


def test_real_out_of_memory_is_reported(dmg):
    # about 1 TB of level arrays: the first allocation already fails
    p = dmg.dmg_default_params(nx=8193, ny=8193, nz=1, h=1.0, batch=2000)
    st, ctx = dmg.dmg_setup(p, torch.ones(1, dtype=torch.float64, device="cuda").data_ptr(),
                            torch.ones(1, dtype=torch.float64, device="cuda").data_ptr())
    assert st == dmg.DMG_ENOMEM and ctx is None


def test_unrolled_work_buffer_failure_keeps_the_context(dmg):
    w = inputs.tissue(17, seed=102)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    q, wv = T(w["q"]), T(w["w"])
    dmg.dmg_debug_fail_alloc(3)
    try:
        st = dmg.dmg_vjp_unrolled(S.ctx, q, wv, 3, 0, None, None, None, None, n=S.n)
    finally:
        dmg.dmg_debug_fail_alloc(0)
    assert st == dmg.DMG_ENOMEM
    u = S.solve(q)
    assert S.last_info.rel_residual <= 1e-10
    u3, qb, Db, mb = S.vjp_unrolled(q, wv, 3)
    assert bool(torch.isfinite(Db).all())
    S.close()
