"""Host-side logic of the request server: slot planning under the memory
budget, the synthetic request stream, and the latency summary (no GPU)."""
import numpy as np

from paper_2608_00760_b300 import serve

SHAPES = [(33, 33, 33), (65, 65, 65), (129, 129, 129), (257, 257, 257), (129, 257, 257)]


def test_plan_slots_respects_budget_and_limits():
    per = {s: 8 * 20 * np.prod(s) for s in SHAPES}          # ~20 FP64 fields per slot
    plan = serve.plan_slots(SHAPES, per, 60e9, max_slots=64)
    assert sum(plan[s] * per[s] for s in SHAPES) <= 60e9 or min(plan.values()) == 1
    assert all(1 <= plan[s] <= 64 and plan[s] * s[0] <= 65535 for s in SHAPES)
    assert plan[(33, 33, 33)] == 64 and plan[(257, 257, 257)] < plan[(129, 129, 129)]
    tiny = serve.plan_slots(SHAPES, per, 1e6)
    assert all(v == 1 for v in tiny.values())


def test_poisson_stream_is_seeded_with_the_requested_mix():
    a = serve.poisson_stream(2000, 200.0, SHAPES, seed=3)
    b = serve.poisson_stream(2000, 200.0, SHAPES, seed=3)
    assert [(r.kind, r.shape, r.arrival) for r in a] == [(r.kind, r.shape, r.arrival) for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0
    kinds = [r.kind for r in a]
    frac = {k: kinds.count(k) / len(kinds) for k in ("fwd", "jvp", "vjp")}
    assert abs(frac["fwd"] - 0.25) < 0.04 and abs(frac["jvp"] - 0.25) < 0.04 and abs(frac["vjp"] - 0.5) < 0.04
    for s in SHAPES:
        assert abs(sum(r.shape == s for r in a) / 2000 - 0.2) < 0.04
    assert sum(r.solves for r in a) == sum({"fwd": 1, "jvp": 2, "vjp": 2}[k] for k in kinds)


def test_summary_latency_and_rates():
    reqs = []
    for i in range(100):
        r = serve.Request(rid=i, kind="vjp", shape=(9, 9, 9), make_inputs=None, arrival=0.01 * i)
        r.t_done = r.arrival + 0.005 + (0.1 if i == 99 else 0.0)
        r.status = 0
        reqs.append(r)
    s = serve.summarize(reqs, 2.0)
    assert s["ok"] == 100 and abs(s["p50_ms"] - 5.0) < 1e-9 and s["p99_ms"] > 5.0
    assert abs(s["seconds"] - (0.99 + 0.105)) < 1e-9
    assert abs(s["solves_per_s"] - 200 / s["seconds"]) < 1e-9
