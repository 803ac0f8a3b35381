"""Continuous-batching request server over the slot-level C ABI (include/dmg.h).

A variational-inference sampler (arXiv 2608.00760, Sec. 2.5) emits forward,
JVP and VJP solves of its samples, each sample with its own coefficients. The
server keeps one pool per grid shape: a batched context whose batch entries are
slots. A request is admitted into a free slot of its shape's pool once the
device-memory budget allows it. Its coefficient hierarchy is built into the slot
(``dmg_slot_load``) and stays resident while it runs its phases:
- forward solve, for every kind;
- then a tangent solve (JVP) or an adjoint solve (VJP), both with the forward
  solution kept in the slot.

Every loop iteration launches one step of every pool with running slots, each on
the pool's own CUDA stream, so pools overlap on the device. Within a pool, all
running slots advance together, one launch per kernel and level (CUDA graphs).
New requests join at any step boundary while older ones are mid-solve (continuous
batching). A slot's arithmetic is that of its sample alone, so each result is bit
for bit the result of the same request served alone.

Latency is measured from a request's arrival to the completion of its last
read-back; the server reports p50/p99 latency beside requests/s and solves/s.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import dmg

class _Cuda:
    """The streams and events the server uses (tests of the scheduling logic
    replace this with a host-only fake)."""

    @staticmethod
    def stream(device):
        import torch
        return torch.cuda.Stream(device)

    @staticmethod
    def use(stream):
        import torch
        return torch.cuda.stream(stream)

    @staticmethod
    def event(stream):
        import torch
        ev = torch.cuda.Event()
        ev.record(stream)
        return ev

    @staticmethod
    def sync(stream):
        stream.synchronize()


_dev = _Cuda()

PHASES = {"fwd": (dmg.DMG_PHASE_FORWARD,),
          "jvp": (dmg.DMG_PHASE_FORWARD, dmg.DMG_PHASE_TANGENT),
          "vjp": (dmg.DMG_PHASE_FORWARD, dmg.DMG_PHASE_ADJOINT)}
# fields a request of each kind brings, and the fields it gets back
INPUT_KEYS = {"fwd": ("D", "mu", "q"), "jvp": ("D", "mu", "q", "dq", "dD", "dmu"),
              "vjp": ("D", "mu", "q", "w")}
OUTPUT_KEYS = {"fwd": ("u",), "jvp": ("u", "du"), "vjp": ("u", "qbar", "Dbar", "mubar")}


@dataclasses.dataclass
class Request:
    """One solve request. ``make_inputs(device)`` returns the float64 tensors of
    INPUT_KEYS[kind] on the device; it is called when the request is admitted,
    on the stream of its pool."""
    rid: int
    kind: str
    shape: tuple
    make_inputs: object
    arrival: float = 0.0
    # filled in by the server
    t_admit: float = None
    t_done: float = None
    status: int = None
    cycles: list = dataclasses.field(default_factory=list)
    rel: list = dataclasses.field(default_factory=list)
    outputs: dict = None
    error: str = None          # why the request failed before it ran (see Server.run)
    pool_steps: tuple = None   # (step of the pool at admission, at completion)

    @property
    def solves(self):
        return len(PHASES[self.kind])

    def io_bytes(self):
        n = int(np.prod(self.shape))
        return 8 * n * (len(INPUT_KEYS[self.kind]) + len(OUTPUT_KEYS[self.kind]))


def coarse_shape(shape):
    """The next level of the grid hierarchy (Sec. 2.2): (n - 1) / 2 + 1 per axis."""
    return tuple((n - 1) // 2 + 1 for n in shape)


def chains(shapes):
    """Group grid shapes into chains of the hierarchy: each next shape is the
    coarse level of the previous one (257^3, 129^3, 65^3, ...). A chain of more
    than one shape is served by one pyramid pool."""
    left = sorted({tuple(s) for s in shapes}, key=lambda s: -int(np.prod(s)))
    out = []
    while left:
        chain = [left.pop(0)]
        while True:
            nxt = coarse_shape(chain[-1])
            if nxt in left:
                left.remove(nxt)
                chain.append(nxt)
            else:
                break
        out.append(chain)
    return out


class Pool:
    """Slots for one grid shape (a context with batch = slots), or for a chain
    of shapes that share their coarse levels (a pyramid context: each level's
    kernels run for the slots of every shape that holds the level)."""

    def __init__(self, shape, h, slots, params, device, chain=None, chain_slots=None):
        import torch
        self.torch = torch
        self.chain = [tuple(s) for s in (chain or [shape])]
        per = [int(x) for x in (chain_slots or [slots])]
        self.shape, self.slots = self.chain[0], sum(per)
        self.n = int(np.prod(self.shape))
        self.device = device
        self.stream = _dev.stream(device)
        nz, ny, nx = self.shape
        if len(self.chain) == 1:
            p = dmg.dmg_default_params(nx=nx, ny=ny, nz=nz, h=float(h), batch=self.slots, **params)
            with _dev.use(self.stream):
                ones = torch.ones((self.slots,) + self.shape, dtype=torch.float64, device=device)
                st, self.ctx = dmg.dmg_setup(p, ones, torch.zeros_like(ones), stream=self.stream)
            del ones
        else:
            p = dmg.dmg_default_params(nx=nx, ny=ny, nz=nz, h=float(h), **params)
            st, self.ctx = dmg.dmg_setup_pyramid(p, per, stream=self.stream)
        _dev.sync(self.stream)
        if st != dmg.DMG_OK:
            raise dmg.DMGError(st, dmg.dmg_last_error(None))
        self.bytes = dmg.dmg_device_bytes(self.ctx)
        # slots of each shape: the pyramid numbers them level by level
        self.free_by = {}
        first = 0
        for s_, k in zip(self.chain, per):
            self.free_by[s_] = list(range(first + k - 1, first - 1, -1))
            first += k
        self.busy = {}        # slot -> [request, phase index, inputs]
        self.steps = 0
        self.step_event = None      # recorded after the launched step's read-back
        self.completing = []        # (event after the read-outs, requests)

    def close(self):
        if self.ctx is not None:
            dmg.dmg_destroy(self.ctx)
            self.ctx = None

    def _check(self, st):
        if st != dmg.DMG_OK:
            raise dmg.DMGError(st, dmg.dmg_last_error(self.ctx))

    @property
    def free(self):
        """Free slots of every shape (the pool can admit when this is not empty)."""
        return [s for v in self.free_by.values() for s in v]

    def has_free(self, shape):
        return bool(self.free_by.get(tuple(shape)))

    def admit(self, req, now):
        """Load the request into a free slot of its shape and stage its forward
        phase. If its inputs cannot be made or the library refuses them, the
        slot goes back to the free list and the exception propagates."""
        free = self.free_by[tuple(req.shape)]
        slot = free.pop()
        n = int(np.prod(req.shape))
        try:
            with _dev.use(self.stream):
                x = req.make_inputs(self.device)
            self._check(dmg.dmg_slot_load(self.ctx, slot, x["D"], x["mu"], self.stream, n=n))
            self._check(dmg.dmg_slot_begin(self.ctx, slot, dmg.DMG_PHASE_FORWARD, x["q"], None, None, self.stream,
                                           n=n))
        except Exception:
            free.append(slot)
            raise
        self.busy[slot] = [req, 0, x]
        req.t_admit = now
        req.pool_steps = (self.steps, None)

    def launch(self):
        self._check(dmg.dmg_step_launch(self.ctx, self.stream))
        self.step_event = _dev.event(self.stream)

    def in_flight(self):
        return self.step_event is not None

    def step_done(self):
        return self.step_event is not None and self.step_event.query()

    def finish(self):
        """Take the finished step: start next phases, enqueue the read-outs of
        requests whose last phase ended and free their slots (later work on the
        pool's stream is ordered after the read-outs)."""
        torch = self.torch
        st, ended = dmg.dmg_step_finish(self.ctx, self.slots, self.stream)
        self.step_event = None
        self._check(st)
        self.steps += 1
        done = []
        for slot in ended:
            entry = self.busy[slot]
            req, ph, x = entry
            n = int(np.prod(req.shape))
            _, status, cyc, rel = dmg.dmg_slot_result(self.ctx, slot)
            req.cycles.append(cyc)
            req.rel.append(rel)
            phases = PHASES[req.kind]
            ok = status in (dmg.DMG_OK,)
            if ok and ph + 1 < len(phases):
                entry[1] = ph + 1
                nxt = phases[ph + 1]
                if nxt == dmg.DMG_PHASE_TANGENT:
                    args = (x["dq"], x["dD"], x["dmu"])
                else:
                    args = (x["w"], None, None)
                self._check(dmg.dmg_slot_begin(self.ctx, slot, nxt, *args, self.stream, n=n))
                continue
            req.status = status
            if ok:
                with _dev.use(self.stream):
                    out = {k: torch.empty(tuple(req.shape), dtype=torch.float64, device=self.device)
                           for k in OUTPUT_KEYS[req.kind]}
                if req.kind == "fwd":
                    self._check(dmg.dmg_slot_read(self.ctx, slot, out["u"], None, None, None, self.stream, n=n))
                elif req.kind == "jvp":
                    self._check(dmg.dmg_slot_read(self.ctx, slot, out["u"], out["du"], None, None, self.stream,
                                                  n=n))
                else:
                    self._check(dmg.dmg_slot_read(self.ctx, slot, out["u"], out["qbar"], out["Dbar"],
                                                  out["mubar"], self.stream, n=n))
                req.outputs = out
            done.append((slot, req))
        if done:
            ev = _dev.event(self.stream)
            for slot, req in done:
                req.pool_steps = (req.pool_steps[0], self.steps)
                self.busy[slot][2] = None
                del self.busy[slot]
                self.free_by[tuple(req.shape)].append(slot)
            self.completing.append((ev, [r for _, r in done]))

    def completed(self, clock):
        """Requests whose read-outs have finished."""
        out = []
        while self.completing and self.completing[0][0].query():
            _, reqs = self.completing.pop(0)
            now = clock()
            for r in reqs:
                r.t_done = now
            out += reqs
        return out

    def active(self):
        return bool(self.busy)

    def idle(self):
        return not self.busy and not self.completing and self.step_event is None


def plan_slots(shapes, per_slot_bytes, pool_budget, max_slots=64):
    """Slots per shape: an equal share of the pool budget each, at most
    max_slots, at least one, and batch * nz <= 65535."""
    share = pool_budget / max(len(shapes), 1)
    plan = {}
    for s in shapes:
        k = int(share // per_slot_bytes[s])
        plan[s] = max(1, min(max_slots, k, 65535 // s[0]))
    return plan


class Server:
    """Pools for the given shapes, sized to the device-memory budget.

    budget_bytes: device memory for the pools and the requests' own tensors;
    pool_fraction of it goes to the pools (slots are fixed at start), the rest
    bounds the inputs and outputs of admitted requests. slots: an explicit
    {shape: slots} plan instead of the budget split. pyramid: shapes that form a
    chain of the grid hierarchy (257^3, 129^3, 65^3, ...) share one pyramid
    pool, whose launches batch the same level across shapes; a chain the
    library refuses (a shape too small to start above the small-level tail)
    falls back to one pool per shape. Off by default: a pyramid steps all its
    slots together, so small requests advance at the rate of the largest grid's
    step, and on the benchmark's mix separate pools (each on its own stream)
    serve more requests per second.
    """

    def __init__(self, shapes, h=0.5, budget_bytes=80e9, params=None, device="cuda", max_slots=64,
                 slots=None, pool_fraction=0.75, pyramid=False):
        params = dict(params or {})
        self.h, self.device = h, device
        self.budget = float(budget_bytes)
        shapes = [tuple(s) for s in shapes]
        if slots is None:
            probe = {}
            for s in shapes:
                p = Pool(s, h, 1, params, device)
                probe[s] = p.bytes
                p.close()
            slots = plan_slots(shapes, probe, pool_fraction * self.budget, max_slots)
        self.slots = {s: slots[s] for s in shapes}
        self.pools = {}
        for chain in (chains(shapes) if pyramid else [[s] for s in shapes]):
            pool = None
            if len(chain) > 1:
                try:
                    pool = Pool(chain[0], h, None, params, device, chain=chain, chain_slots=[slots[s] for s in chain])
                except dmg.DMGError:
                    pool = None
            if pool is not None:
                for s in chain:
                    self.pools[s] = pool
            else:
                for s in chain:
                    self.pools[s] = Pool(s, h, slots[s], params, device)
        self.pool_bytes = sum(p.bytes for p in self.unique_pools())
        if self.pool_bytes > self.budget:
            raise ValueError("pools need %.1f GB, above the budget of %.1f GB" % (self.pool_bytes / 1e9,
                                                                                   self.budget / 1e9))
        self.io_bytes = 0

    def unique_pools(self):
        out = []
        for p in self.pools.values():
            if all(p is not q for q in out):
                out.append(p)
        return out

    def close(self):
        for p in self.unique_pools():
            p.close()

    def _admit(self, queue, now):
        """FIFO per shape: the oldest waiting request of each shape is admitted
        when its pool has a free slot and its tensors fit the budget; a full
        pool does not hold back requests of other shapes. Returns the requests
        that failed at admission (their inputs could not be made, or the
        library refused them): they end at once with a status and a message,
        and the others go on."""
        blocked = set()
        kept = collections.deque()
        failed = []
        while queue:
            req = queue.popleft()
            pool = self.pools[tuple(req.shape)]
            need = req.io_bytes()
            if (req.shape in blocked or not pool.has_free(req.shape) or
                    self.pool_bytes + self.io_bytes + need > self.budget):
                blocked.add(req.shape)
                kept.append(req)
                continue
            try:
                pool.admit(req, now)
            except Exception as e:   # noqa: BLE001 - one request's failure is reported, not raised
                req.status = e.status if isinstance(e, dmg.DMGError) else dmg.DMG_EINVAL
                req.error = "%s: %s" % (type(e).__name__, e)
                req.t_admit = req.t_done = now
                failed.append(req)
                continue
            self.io_bytes += need
        queue.extend(kept)
        return failed

    def run(self, requests, realtime=True, keep_outputs=True):
        """Serve the requests (arrival times in seconds from the start). With
        realtime=False every request is available at once; keep_outputs=False
        drops each result once it has been read back. Returns the served
        requests and summary statistics."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue = collections.deque()
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0
        served = []
        pools = self.unique_pools()
        while pending or queue or not all(p.idle() for p in pools):
            now = clock()
            while pending and (not realtime or pending[0].arrival <= now):
                queue.append(pending.popleft())
            served += self._admit(queue, now)
            # each pool advances on its own: a finished step is taken and the
            # next one launched at once, so pools with short steps do not wait
            # for pools with long ones
            moved = False
            for p in pools:
                if p.step_done():
                    p.finish()
                    # slots freed by this step take waiting requests before the
                    # next step is launched, so they lose no step
                    served += self._admit(queue, clock())
                    moved = True
                if not p.in_flight() and p.active():
                    p.launch()
                    moved = True
                for req in p.completed(clock):
                    self.io_bytes -= req.io_bytes()
                    if not keep_outputs:
                        req.outputs = None
                    served.append(req)
                    moved = True
            if moved:
                continue
            if all(p.idle() for p in pools):
                if queue:
                    raise ValueError("request %d (%s) does not fit the memory budget even alone"
                                     % (queue[0].rid, "x".join(map(str, queue[0].shape[::-1]))))
                if pending:
                    time.sleep(max(0.0, pending[0].arrival - clock()))
            else:
                time.sleep(2e-5)
        return served, summarize(served, clock())


def summarize(served, wall):
    """Rates over the requests that ended with DMG_OK; latency percentiles over
    those requests too (arrival to the end of the read-back)."""
    ok = [r for r in served if r.status == dmg.DMG_OK]
    lat = [1e3 * (r.t_done - r.arrival) for r in ok if r.t_done is not None]
    first = min((r.arrival for r in served), default=0.0)
    last = max((r.t_done for r in served if r.t_done is not None), default=wall)
    span = max(last - first, 1e-9)
    return dict(requests=len(served), ok=len(ok), seconds=span,
                requests_per_s=len(ok) / span, solves_per_s=sum(r.solves for r in ok) / span,
                p50_ms=float(np.percentile(lat, 50)) if lat else None,
                p99_ms=float(np.percentile(lat, 99)) if lat else None)


def poisson_stream(n, rate, shapes, mix=(("fwd", 1), ("jvp", 1), ("vjp", 2)), seed=0, h=0.5):
    """n requests with exponential inter-arrival times of mean 1/rate, shapes
    drawn uniformly, kinds by the weights of mix, inputs from the tissue recipe
    with a per-request seed (drawn on the device when the request is admitted)."""
    from . import inputs
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    kinds = [k for k, _ in mix]
    wts = np.array([w for _, w in mix], dtype=float)
    reqs = []
    for i in range(n):
        shape = tuple(shapes[rng.integers(len(shapes))])
        kind = kinds[rng.choice(len(kinds), p=wts / wts.sum())]
        rseed = int(rng.integers(1 << 62))

        def make(device, shape=shape, kind=kind, rseed=rseed):
            return inputs.tissue_torch(shape, rseed, h=h, device=device, keys=INPUT_KEYS[kind])

        reqs.append(Request(rid=i, kind=kind, shape=shape, make_inputs=make, arrival=float(t[i])))
    return reqs


def run_alone(req, h=0.5, params=None, device="cuda"):
    """The request on its own: a context of batch 1, the whole-context calls."""
    import torch
    x = req.make_inputs(device)
    S = dmg.Solver(x["D"], x["mu"], h, **(params or {}))
    try:
        u = S.solve(x["q"])
        if req.kind == "fwd":
            return {"u": u}
        if req.kind == "jvp":
            return {"u": u, "du": S.jvp(u, x["dq"], x["dD"], x["dmu"])}
        qb, Db, mb = S.vjp(u, x["w"])
        return {"u": u, "qbar": qb, "Dbar": Db, "mubar": mb}
    finally:
        S.close()


def run_one_at_a_time(requests, h=0.5, params=None, device="cuda"):
    """Every request alone and in arrival order (setup, solves, read-back);
    returns the wall time in seconds."""
    import torch
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        out = run_alone(r, h, params, device)
        del out
    torch.cuda.synchronize(device)
    return time.perf_counter() - t0
