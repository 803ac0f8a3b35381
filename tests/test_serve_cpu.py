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


# ---------------------------------------------------------------------------
# The scheduler itself, run on the host against a fake of the slot-level C ABI.
# The fake keeps the contract of include/dmg.h's slot calls: a slot is loaded,
# begins a phase, every step advances every running slot by one cycle, and
# dmg_step_finish reports the slots whose phase ended in that step. Here a
# phase ends after as many steps as the first entry of its right-hand side
# (a negative value ends it unconverged), and dmg_slot_read writes constants
# that say which input each output came from, so routing mistakes show.

import contextlib
import types

import pytest
import torch

from paper_2608_00760_b300 import dmg as real_dmg


class FakeABI:
    def __init__(self, per_slot_bytes=1000):
        for k in dir(real_dmg):
            if k.startswith("DMG_"):
                setattr(self, k, getattr(real_dmg, k))
        self.DMGError = real_dmg.DMGError
        self.per_slot_bytes = per_slot_bytes
        self.launches = 0
        self.admissions = []          # (rid-like tag from D, slot) in admission order
        self.max_running = 0

    # context ---------------------------------------------------------------
    def dmg_default_params(self, **kw):
        return types.SimpleNamespace(**kw)

    def dmg_setup(self, p, D, mu, stream=None):
        assert D.shape == (p.batch, p.nz, p.ny, p.nx)
        ctx = types.SimpleNamespace(batch=p.batch, slots=[None] * p.batch, in_flight=False, closed=False)
        return self.DMG_OK, ctx

    def dmg_device_bytes(self, ctx):
        return self.per_slot_bytes * ctx.batch

    def dmg_destroy(self, ctx):
        ctx.closed = True
        return self.DMG_OK

    def dmg_last_error(self, ctx=None):
        return "fake"

    # slots -----------------------------------------------------------------
    def dmg_slot_load(self, ctx, slot, D, mu, stream=None, n=None):
        sl = ctx.slots[slot]
        assert sl is None or sl["left"] == 0, "load into a running slot"
        ctx.slots[slot] = dict(D=float(D.flatten()[0]), mu=float(mu.flatten()[0]), phase=None, left=0,
                               status=None, cycles=0, val={})
        self.admissions.append((int(D.flatten()[0]), slot))
        return self.DMG_OK

    def dmg_slot_begin(self, ctx, slot, phase, a=None, b=None, c=None, stream=None, n=None):
        sl = ctx.slots[slot]
        # a phase may be staged while a step is in flight; it joins from the next launch
        assert sl is not None and sl["left"] == 0
        if phase != self.DMG_PHASE_FORWARD:
            assert sl["status"] == self.DMG_OK and sl["phase"] == self.DMG_PHASE_FORWARD
        v = float(a.flatten()[0])
        sl.update(phase=phase, left=int(abs(v)), status=self.DMG_OK if v > 0 else self.DMG_ENOCONV, cycles=0)
        sl["val"][phase] = v
        return self.DMG_OK

    def dmg_step_launch(self, ctx, stream=None):
        assert not ctx.in_flight, "a second step launched before the first was finished"
        running = [s for s in ctx.slots if s is not None and s["left"] > 0]
        assert running, "a step launched with no running slot"
        self.max_running = max(self.max_running, len(running))
        for s in running:
            s["left"] -= 1
            s["cycles"] += 1
            s["ended_now"] = s["left"] == 0
        ctx.in_flight = True
        self.launches += 1
        return self.DMG_OK

    def dmg_step_finish(self, ctx, batch, stream=None):
        assert ctx.in_flight
        ctx.in_flight = False
        ended = []
        for i, s in enumerate(ctx.slots):
            if s is not None and s.pop("ended_now", False):
                ended.append(i)
        return self.DMG_OK, ended

    def dmg_slot_result(self, ctx, slot):
        s = ctx.slots[slot]
        return self.DMG_OK, (-1 if s["left"] else s["status"]), s["cycles"], 1e-11

    def dmg_slot_read(self, ctx, slot, u=None, x=None, Dbar=None, mubar=None, stream=None, n=None):
        s = ctx.slots[slot]
        assert s["left"] == 0 and s["status"] == self.DMG_OK
        u.fill_(10 * s["val"][self.DMG_PHASE_FORWARD])
        if x is not None:
            x.fill_(10 * s["val"][s["phase"]])
        if Dbar is not None:
            Dbar.fill_(s["D"])
            mubar.fill_(s["mu"])
        return self.DMG_OK


class FakeEvent:
    """Completes after `lag` queries (device work still running before that)."""

    def __init__(self, lag):
        self.left = lag

    def query(self):
        self.left -= 1
        return self.left < 0


class FakeDevice:
    def __init__(self, lag=0):
        self.lag = lag

    def stream(self, device):
        return object()

    def use(self, stream):
        return contextlib.nullcontext()

    def event(self, stream):
        return FakeEvent(self.lag)

    def sync(self, stream):
        pass


@pytest.fixture
def fake(monkeypatch):
    def install(lag=0, per_slot_bytes=1000):
        abi = FakeABI(per_slot_bytes)
        monkeypatch.setattr(serve, "dmg", abi)
        monkeypatch.setattr(serve, "_dev", FakeDevice(lag))
        return abi
    return install


def req(rid, kind, shape, steps, arrival=0.0):
    """steps: forward steps, then tangent or adjoint steps (negative: unconverged)."""
    def make(device):
        f = lambda v: torch.full(shape, float(v), dtype=torch.float64, device=device)
        x = {"D": f(rid), "mu": f(rid + 0.5), "q": f(steps[0])}
        if kind == "jvp":
            x.update(dq=f(steps[1]), dD=f(0), dmu=f(0))
        if kind == "vjp":
            x["w"] = f(steps[1])
        return x
    return serve.Request(rid=rid, kind=kind, shape=shape, make_inputs=make, arrival=arrival)


S1, S2 = (5, 5, 5), (9, 5, 5)


@pytest.mark.parametrize("lag", [0, 3])
def test_phases_chain_without_idle_steps_and_outputs_are_routed(fake, lag):
    abi = fake(lag=lag)
    srv = serve.Server([S1], budget_bytes=1e9, device="cpu", slots={S1: 4})
    reqs = [req(1, "fwd", S1, (3,)), req(2, "jvp", S1, (2, 5)), req(3, "vjp", S1, (4, 1)),
            req(4, "vjp", S1, (1, 6))]
    served, summ = srv.run(reqs, realtime=False)
    assert sorted(r.rid for r in served) == [1, 2, 3, 4] and summ["ok"] == 4
    by = {r.rid: r for r in served}
    for rid, steps in ((1, (3,)), (2, (2, 5)), (3, (4, 1)), (4, (1, 6))):
        r = by[rid]
        assert r.status == real_dmg.DMG_OK and r.cycles == list(steps)
        # a follow-up phase starts in the step right after the forward solve ends
        assert r.pool_steps[1] - r.pool_steps[0] == sum(steps)
        assert torch.all(r.outputs["u"] == 10 * steps[0])
        assert r.t_done is not None and r.t_done >= r.t_admit
    assert torch.all(by[2].outputs["du"] == 50)
    assert torch.all(by[3].outputs["qbar"] == 10) and torch.all(by[3].outputs["Dbar"] == 3)
    assert torch.all(by[3].outputs["mubar"] == 3.5)
    assert set(by[4].outputs) == {"u", "qbar", "Dbar", "mubar"} and set(by[1].outputs) == {"u"}
    # all four run together: the step count is the longest request's
    assert abi.launches == 7 and abi.max_running == 4
    srv.close()
    assert srv.pools[S1].ctx is None


def test_unconverged_phase_ends_the_request_and_frees_its_slot(fake):
    abi = fake()
    srv = serve.Server([S1], budget_bytes=1e9, device="cpu", slots={S1: 1})
    reqs = [req(1, "jvp", S1, (-2, 4)), req(2, "vjp", S1, (3, -1)), req(3, "fwd", S1, (1,))]
    served, summ = srv.run(reqs, realtime=False, keep_outputs=True)
    by = {r.rid: r for r in served}
    assert by[1].status == real_dmg.DMG_ENOCONV and by[1].cycles == [2] and by[1].outputs is None
    assert by[2].status == real_dmg.DMG_ENOCONV and by[2].cycles == [3, 1] and by[2].outputs is None
    assert by[3].status == real_dmg.DMG_OK and torch.all(by[3].outputs["u"] == 10)
    assert summ["ok"] == 1 and summ["requests"] == 3
    # one slot: the requests ran one after another through it
    assert [s for _, s in abi.admissions] == [0, 0, 0]
    assert abi.launches == 2 + 4 + 1


def test_fifo_per_shape_and_a_full_pool_does_not_block_other_shapes(fake):
    abi = fake()
    srv = serve.Server([S1, S2], budget_bytes=1e9, device="cpu", slots={S1: 1, S2: 2})
    reqs = [req(1, "fwd", S1, (5,), 0.0), req(2, "fwd", S1, (1,), 0.1), req(3, "fwd", S2, (2,), 0.2),
            req(4, "fwd", S2, (2,), 0.3), req(5, "fwd", S1, (1,), 0.4), req(6, "fwd", S2, (1,), 0.5)]
    served, _ = srv.run(reqs, realtime=False)
    order = [rid for rid, _ in abi.admissions]
    # shape S1 admits in arrival order, and so does S2
    assert [r for r in order if r in (1, 2, 5)] == [1, 2, 5]
    assert [r for r in order if r in (3, 4, 6)] == [3, 4, 6]
    # S2's requests are admitted while request 2 waits for S1's only slot
    assert order[:3] == [1, 3, 4]
    by = {r.rid: r for r in served}
    assert by[2].pool_steps[0] == 5 and by[5].pool_steps[0] == 6
    assert all(r.status == real_dmg.DMG_OK for r in served)


def test_continuous_batching_admits_into_a_running_pool(fake):
    fake()
    srv = serve.Server([S1], budget_bytes=1e9, device="cpu", slots={S1: 2})
    reqs = [req(1, "fwd", S1, (6,)), req(2, "fwd", S1, (1,)), req(3, "vjp", S1, (2, 2))]
    served, _ = srv.run(reqs, realtime=False)
    by = {r.rid: r for r in served}
    # request 3 takes the slot request 2 freed while request 1 is mid-solve
    assert by[1].pool_steps == (0, 6) and by[2].pool_steps == (0, 1)
    assert by[3].pool_steps == (1, 5)


def test_memory_budget_bounds_the_admitted_requests(fake, monkeypatch):
    fake(per_slot_bytes=1000)
    io = req(0, "vjp", S1, (1, 1)).io_bytes()             # 8 * 125 * 8 bytes
    # pools take 4000 bytes; room for exactly two vjp requests' tensors
    srv = serve.Server([S1], budget_bytes=4000 + 2 * io + io // 2, device="cpu", slots={S1: 4})
    peak = [0]
    admit = serve.Server._admit

    def tracking(self, queue, now):
        out = admit(self, queue, now)
        peak[0] = max(peak[0], self.io_bytes)
        assert self.pool_bytes + self.io_bytes <= self.budget
        return out

    monkeypatch.setattr(serve.Server, "_admit", tracking)
    served, summ = srv.run([req(i, "vjp", S1, (2, 2)) for i in range(1, 7)], realtime=False)
    assert summ["ok"] == 6 and peak[0] == 2 * io and srv.io_bytes == 0
    # with room for two, six requests of four steps each take three rounds
    assert max(r.pool_steps[1] for r in served) == 12


def test_a_request_larger_than_the_budget_is_refused(fake):
    fake(per_slot_bytes=1000)
    big = (33, 33, 33)
    srv = serve.Server([big], budget_bytes=1000 + 1000, device="cpu", slots={big: 1})
    with pytest.raises(ValueError, match="does not fit the memory budget"):
        srv.run([req(1, "fwd", big, (1,))], realtime=False)


def test_pools_are_sized_from_the_probed_slot_bytes(fake):
    fake(per_slot_bytes=10_000)
    srv = serve.Server([S1, S2], budget_bytes=1e5, device="cpu", max_slots=64, pool_fraction=0.8)
    # 80 kB for pools split evenly: 40 kB each, 10 kB per slot -> 4 slots
    assert srv.pools[S1].slots == 4 and srv.pools[S2].slots == 4 and srv.pool_bytes == 80_000


def test_realtime_arrivals_and_dropped_outputs(fake):
    fake(lag=1)
    srv = serve.Server([S1], budget_bytes=1e9, device="cpu", slots={S1: 2})
    reqs = [req(i, "fwd", S1, (1 + i % 3,), arrival=0.002 * i) for i in range(10)]
    served, summ = srv.run(reqs, realtime=True, keep_outputs=False)
    assert summ["ok"] == 10 and all(r.outputs is None for r in served)
    assert all(r.t_admit >= r.arrival and r.t_done > r.t_admit for r in served)
    assert summ["p50_ms"] > 0 and summ["p99_ms"] >= summ["p50_ms"]


def test_a_request_that_fails_at_admission_ends_alone(fake):
    abi = fake()
    srv = serve.Server([S1], budget_bytes=1e9, device="cpu", slots={S1: 2})

    def broken(device):
        raise RuntimeError("no such sample")

    bad = serve.Request(rid=9, kind="fwd", shape=S1, make_inputs=broken, arrival=0.0)
    reqs = [req(1, "vjp", S1, (2, 2)), bad, req(2, "fwd", S1, (3,)), req(3, "jvp", S1, (1, 1))]
    served, summ = srv.run(reqs, realtime=False)
    by = {r.rid: r for r in served}
    assert set(by) == {1, 2, 3, 9}
    assert by[9].status == real_dmg.DMG_EINVAL and "no such sample" in by[9].error and by[9].outputs is None
    assert all(by[r].status == real_dmg.DMG_OK and by[r].error is None for r in (1, 2, 3))
    assert summ["ok"] == 3 and summ["requests"] == 4
    # the slot it was offered went back to the pool, and its bytes were never counted
    pool = srv.pools[S1]
    assert sorted(pool.free) == [0, 1] and not pool.busy and srv.io_bytes == 0
    assert [rid for rid, _ in abi.admissions] == [1, 2, 3]


def test_a_refused_slot_load_ends_that_request_with_the_library_status(fake, monkeypatch):
    abi = fake()
    load = abi.dmg_slot_load

    def refusing(ctx, slot, D, mu, stream=None, n=None):
        if float(D.flatten()[0]) == 7.0:
            return abi.DMG_ENOMEM
        return load(ctx, slot, D, mu, stream, n)

    monkeypatch.setattr(abi, "dmg_slot_load", refusing)
    srv = serve.Server([S1], budget_bytes=1e9, device="cpu", slots={S1: 1})
    served, summ = srv.run([req(7, "fwd", S1, (2,)), req(8, "fwd", S1, (2,))], realtime=False)
    by = {r.rid: r for r in served}
    assert by[7].status == real_dmg.DMG_ENOMEM and by[7].error.startswith("DMGError")
    assert by[8].status == real_dmg.DMG_OK and by[8].pool_steps == (0, 2)
    assert summ["ok"] == 1 and summ["p50_ms"] is not None


def test_chains_group_shapes_of_one_hierarchy():
    from paper_2608_00760_b300 import serve
    shapes = [(33, 33, 33), (65, 65, 65), (129, 129, 129), (257, 257, 257), (129, 257, 257)]
    assert serve.chains(shapes) == [[(257, 257, 257), (129, 129, 129), (65, 65, 65), (33, 33, 33)],
                                    [(129, 257, 257)]]
    assert serve.chains([(17, 17, 17), (9, 17, 33)]) == [[(9, 17, 33)], [(17, 17, 17)]]
    assert serve.coarse_shape((257, 257, 129)) == (129, 129, 65)
