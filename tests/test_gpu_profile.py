"""The instrumentation the benchmark's roofline numbers come from:
dmg_profile_begin/end count the launches of one kernel on one level inside the
replayed graphs and sum their event-timed durations. Checked through the C ABI
on the three level-0 schedules of a V(2,2) cycle:
  - FP64: 4 pre + 4 post half-sweeps and one prolongation per cycle;
  - FP32, fused levels (fewer than 2^22 vertices): 4 pre half-sweeps, the
    prolongation fused into the first post half-sweep (counted as PROLONG),
    then 3 more half-sweeps;
  - FP32, split levels: 4 pre half-sweeps, the one-colour correction (PROLONG),
    then 4 post half-sweeps.
Profiling only adds event nodes: the results stay bit for bit those of an
unprofiled run."""
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


def profiled(dmg, S, kernel, fp32, run):
    assert dmg.dmg_profile_begin(S.ctx, kernel, 0, fp32) == dmg.DMG_OK
    out = run()
    st, n, ms = dmg.dmg_profile_end(S.ctx)
    assert st == dmg.DMG_OK
    return out, n, ms


def test_fp64_fixed_cycles_counts(dmg):
    w = inputs.tissue(65, seed=60)
    m = 3
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], fixed_cycles=m)
    q = T(w["q"])
    ref = S.solve(q).clone()
    u, n, ms = profiled(dmg, S, dmg.DMG_KERNEL_SMOOTH, False, lambda: S.solve(q))
    assert n == 8 * m and 0 < ms / n < 5.0
    assert torch.equal(u, ref)
    _, n, ms = profiled(dmg, S, dmg.DMG_KERNEL_PROLONG, False, lambda: S.solve(q))
    assert n == m and ms > 0
    S.close()


def test_direct_launches_are_timed(dmg):
    # the gradient kernel runs outside the captured graphs: its events are plain records
    w = inputs.tissue(33, seed=63)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    u = S.solve(T(w["q"]))
    ref = S.vjp(u, T(w["w"]))
    out, n, ms = profiled(dmg, S, dmg.DMG_KERNEL_GRAD, False, lambda: S.vjp(u, T(w["w"])))
    assert n == 1 and ms > 0
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    # the tail (inside the graphs) is counted on its first level only, once per V-cycle
    q = T(w["q"])
    S.solve(q)
    cycles = S.last_info.cycles
    counts = []
    for lev in range(dmg.dmg_levels(S.ctx)):
        assert dmg.dmg_profile_begin(S.ctx, dmg.DMG_KERNEL_TAIL, lev, 0) == dmg.DMG_OK
        S.solve(q)
        st, n, ms = dmg.dmg_profile_end(S.ctx)
        assert st == dmg.DMG_OK and (n == 0 or ms > 0)
        counts.append(n)
    assert sorted(counts)[-1] == cycles and sum(counts) == cycles
    S.close()


def test_mixed_fused_level_counts(dmg):
    w = inputs.tissue(65, seed=61)   # 65^3: a fused level
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=dmg.DMG_MIXED)
    q = T(w["q"])
    ref = S.solve(q).clone()
    cycles = S.last_info.cycles
    u, n, ms = profiled(dmg, S, dmg.DMG_KERNEL_SMOOTH, True, lambda: S.solve(q))
    assert S.last_info.cycles == cycles
    assert n == 7 * cycles and 0 < ms / n < 5.0
    assert torch.equal(u, ref)
    _, n, ms = profiled(dmg, S, dmg.DMG_KERNEL_PROLONG, True, lambda: S.solve(q))
    assert n == cycles and ms > 0
    S.close()


def test_mixed_split_level_counts(dmg):
    # two copies of one 129^3 problem: 2 x 129 x 129 x 192 padded vertices >= 2^22, a split level;
    # both samples converge at the same step, so every launch serves both
    w = inputs.tissue(129, seed=62)
    st = lambda k: T(np.stack([w[k], w[k]]))
    S = dmg.Solver(st("D"), st("mu"), w["h"], precision=dmg.DMG_MIXED)
    q = st("q")
    ref = S.solve(q).clone()
    cycles = S.last_info.cycles
    assert torch.equal(ref[0], ref[1])
    u, n, ms = profiled(dmg, S, dmg.DMG_KERNEL_SMOOTH, True, lambda: S.solve(q))
    assert n == 8 * cycles and 0 < ms / n < 5.0
    assert torch.equal(u, ref)
    _, n, ms = profiled(dmg, S, dmg.DMG_KERNEL_PROLONG, True, lambda: S.solve(q))
    assert n == cycles and ms > 0
    # the same problem alone (129 x 129 x 192 < 2^22: fused) ends bitwise alike
    A = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=dmg.DMG_MIXED)
    assert torch.equal(A.solve(T(w["q"])), ref[0])
    S.close()
    A.close()
