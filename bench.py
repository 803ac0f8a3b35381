#!/usr/bin/env python3
"""Benchmark: forward solve + VJP (w.r.t. q, D, mu) pairs per second on the
257^3 tissue-like workload at relative residual 1e-10, mixed precision (FP32
inner V-cycles, FP64 defect correction) and plain FP64, on one B300 per rank.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dmg|reference]

One step = dmg_solve(q) followed by dmg_vjp(u, w) returning (qbar, Dbar, mubar),
both converged to relative residual 1e-10. The coefficient hierarchy
(dmg_setup) is built once, outside the timed region: the coefficients are fixed
while sources vary, as in the paper's inference use. Every field is 136 MB in
FP64, larger than the 126 MB L2, so no L2 flush is needed between steps.

The line also carries ``serving``: a stream of 2000 Poisson-arrival forward,
JVP and VJP requests at 200/s on five grid shapes, served with continuous
batching under an 80 GB budget (p50/p99 latency, solves/s), next to the same
requests run one at a time in FP64. And ``vi_batch``: the batched variational-inference step,
64 tissue samples of 129^3 (each with its own coefficients, source and
cotangent) solved forward and pulled back together in one context (one launch
per kernel and level for all samples), in samples/s, next to the same samples
run one at a time.

Multi-GPU: a single solve does not shard, so N ranks run N independent replicas
(weak scaling); the timed region is bracketed by barriers and the max over
ranks is reported. --impl reference times the FP64 CPU oracle on this host's
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+VJP solves/s & HBM GB/s at 257³ (FP32-refined vs FP64, 1e-10); p50/p99"
UNIT = "fwd+VJP solves/s"
N_SIDE = 257
RTOL = 1e-10
# Roofline unit: one RB-GS half-sweep launch on the finest level (one colour).
# Algorithmic bytes: a full FP32 red-black sweep must read
# u, f, D and mu once and write u once, 20 B per interior vertex, so one
# half-sweep is charged 10 B per interior vertex of the grid. The kernel as
# built moves 12 B per vertex per half-sweep (f and mu of its own colour,
# D of every vertex, u of the other colour, u written on its own colour); the
# line reports the fraction in both units.
# FP64 (precomputed faces): 6 FMA + 1 MUL per updated vertex = 3.5 FP64-pipe
# operations per interior vertex of the grid, against the FP64 FMA rate that
# dmg_probe_fma measures on the device at the start of the run.
HALF_SWEEP_BYTES_FP32 = 10.0
HALF_SWEEP_BYTES_FP32_KERNEL = 12.0
HALF_SWEEP_FP64_OPS = 3.5
# DRAM bytes (read + write) of one finest-level half-sweep launch at 257^3,
# from an ncu capture of the current kernel
HALF_SWEEP_TRAFFIC = {"fp32": 208017152, "fp64": 664092672}
# DRAM bytes per sample of one batched finest-level FP32 half-sweep at 129^3,
# from an ncu capture of 8 samples, scaled by the sample count (None: the
# kernel changed since the last capture)
VI_HALF_SWEEP_TRAFFIC_PER_SAMPLE_129 = 28567808


AUTOTUNE = [1]   # set from --autotune
TWIN = [1]       # set from --twin


def percentile(x, p):
    return float(np.percentile(np.asarray(x), p)) if len(x) else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "dmg_clocks_%d_%d.csv" % (os.getpid(), index))

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), power=float(f[3]), hw=f[5], hwt=f[6],
                                 swt=f[7], swp=f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in rows])), "sm_max_mhz": max(r["smax"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# FP64 FMA rate (FMA instructions per second) of the device, measured by
# dmg_probe_fma at the start of every run (main()); the denominator of the FP64
# kernels' roofline
FP64_OPS_PEAK = [None]


def host_info():
    """The host's core count (all, and usable by this process) and CPU model."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except Exception:
        pass
    try:
        usable = len(os.sched_getaffinity(0))
    except Exception:
        usable = os.cpu_count()
    return dict(nproc=os.cpu_count(), usable=usable, cpu_model=model)


def make_inputs(n, seed=0):
    from paper_2608_00760_b300 import inputs
    return inputs.tissue(n, seed=seed)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, max_total_ms):
    """Whole-job pairs/s: every rank runs `steps` pairs; the slowest rank's time counts."""
    return world * steps / (max_total_ms / 1e3)


def profiled_pass(dmg, torch, S, step, steps, kernel, fp32, stream, dev):
    """Launch durations of one kernel on level 0, from CUDA event nodes around
    each of its launches inside the replayed graphs, over a pass of `steps`
    more steps after the timed one (the event nodes cost time of their own, so
    they stay out of the timed pass). Returns launches, their total ms and the
    pass's ms per step (the first, untimed step re-captures the graphs)."""
    dmg.dmg_profile_begin(S.ctx, kernel, 0, fp32, max_launches=4096)
    step()
    torch.cuda.synchronize(dev)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize(dev)
    _, n, ms = dmg.dmg_profile_end(S.ctx)
    return dict(launches=n, total_ms=ms, pass_ms_per_step=p0.elapsed_time(p1) / steps)


def run_arm(dmg, torch, w, precision, steps, warmup, world, local, profile=None, clocks=False, inner=1):
    """Times `steps` fwd+VJP pairs; returns a result dict."""
    dev = torch.device("cuda", local)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    D, mu, q, wv = T(w["D"]), T(w["mu"]), T(w["q"]), T(w["w"])
    S = dmg.Solver(D, mu, w["h"], precision=precision, rtol=RTOL, inner_cycles=inner, autotune=AUTOTUNE[0],
                   twin_adjoint=TWIN[0])
    u = torch.empty_like(q)
    qb, Db, mb = torch.empty_like(q), torch.empty_like(q), torch.empty_like(q)
    info_f, info_a = dmg.dmg_info(), dmg.dmg_info()
    stream = torch.cuda.current_stream(dev)

    def step():
        # one pair through the pair call: the adjoint solve runs beside the
        # forward one (twin_adjoint, the default)
        st = dmg.dmg_solve_vjp(S.ctx, q, wv, u, qb, Db, mb, info_f, info_a, stream, n=S.n)
        if st != dmg.DMG_OK:
            raise dmg.DMGError(st, dmg.dmg_last_error(S.ctx))

    def step_seq():
        # the same pair as two calls, one solve after the other
        st = dmg.dmg_solve(S.ctx, q, u, info_f, stream, n=S.n)
        if st != dmg.DMG_OK:
            raise dmg.DMGError(st, dmg.dmg_last_error(S.ctx))
        st = dmg.dmg_vjp(S.ctx, u, wv, 0, qb, Db, mb, info_a, stream, n=S.n)
        if st != dmg.DMG_OK:
            raise dmg.DMGError(st, dmg.dmg_last_error(S.ctx))

    for _ in range(warmup):
        step()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    l0 = dmg.dmg_launch_count(S.ctx)
    barrier(world)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local) if clocks else None
    if sampler:
        sampler.__enter__()
    ev[0].record(stream)
    for i in range(steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.__exit__()
    barrier(world)
    launches = dmg.dmg_launch_count(S.ctx) - l0
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total_ms = ev[0].elapsed_time(ev[steps])
    prof = None
    seq_ms = None
    if profile is not None:
        # kernel durations from the two-call form: no second lane competes for
        # the GPU while the profiled kernel runs
        for _ in range(2):
            step_seq()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step_seq()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        seq_ms = e0.elapsed_time(e1) / steps
        prof = profiled_pass(dmg, torch, S, step_seq, steps, profile[0], profile[1], stream, dev)
    res = dict(total_ms=max_over_ranks(world, total_ms), per_ms=per, launches=launches,
               fwd_cycles=info_f.cycles, fwd_outer=info_f.outer, adj_cycles=info_a.cycles,
               adj_outer=info_a.outer, fwd_rel=info_f.rel_residual, adj_rel=info_a.rel_residual,
               prof=prof, seq_ms=seq_ms, clocks=sampler.summary() if sampler else None, solver=S,
               out=(u, qb, Db, mb))
    return res


def run_e2e(dmg, torch, w, precision, steps, warmup, world, local, inner=1):
    """Same pairs through the C ABI with pinned HOST buffers. Streamed: one
    dmg_solve_vjp_many call for all `steps` pairs, each pair's q, w copied
    host->device and u, qbar, Dbar, mubar device->host inside the call (two
    distinct pinned input and output sets, alternating between pairs, so every
    pair moves its own bytes), with the transfers overlapped with the
    neighbouring pairs' solves. Single: one dmg_solve_vjp call per pair.
    Device stream: one dmg_solve_vjp_many call over device-resident inputs and
    outputs (two sets, alternating), so that only the overlap of a pair's
    gradient and read-out with the next pair's solves differs from the
    headline's one call per pair."""
    dev = torch.device("cuda", local)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision, rtol=RTOL, inner_cycles=inner)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    qh = [pin(w["q"]), pin(w["q"] * 1.5)]
    wh = [pin(w["w"]), pin(-w["w"])]
    outs = [[torch.empty(w["shape"], dtype=torch.float64).pin_memory() for _ in range(2)] for _ in range(4)]
    stream = torch.cuda.current_stream(dev)

    def many(k):
        st = dmg.dmg_solve_vjp_many(S.ctx, [qh[i % 2] for i in range(k)], [wh[i % 2] for i in range(k)],
                                    *[[o[i % 2] for i in range(k)] for o in outs], stream=stream, n=S.n)
        assert st == dmg.DMG_OK, dmg.dmg_last_error(S.ctx)

    def single():
        st = dmg.dmg_solve_vjp(S.ctx, qh[0], wh[0], outs[0][0], outs[1][0], outs[2][0], outs[3][0], None, None,
                               stream, n=S.n)
        assert st == dmg.DMG_OK, dmg.dmg_last_error(S.ctx)

    qd, wd = [T(w["q"]), T(w["q"] * 1.5)], [T(w["w"]), T(-w["w"])]
    outd = [[torch.empty(w["shape"], dtype=torch.float64, device=dev) for _ in range(2)] for _ in range(4)]

    def many_device(k):
        st = dmg.dmg_solve_vjp_many(S.ctx, [qd[i % 2] for i in range(k)], [wd[i % 2] for i in range(k)],
                                    *[[o[i % 2] for i in range(k)] for o in outd], stream=stream, n=S.n)
        assert st == dmg.DMG_OK, dmg.dmg_last_error(S.ctx)

    many(2)   # allocates the staging buffers, warms up
    many_device(2)
    for _ in range(warmup):
        single()
    res = {}
    for name, fn in (("streamed", lambda: many(steps)), ("single", lambda: [single() for _ in range(steps)]),
                     ("device", lambda: many_device(steps))):
        barrier(world)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        barrier(world)
        res[name] = max_over_ranks(world, el)
    nbytes = 8 * int(np.prod(w["shape"]))
    S.close()
    return dict(seconds=res["streamed"], seconds_single=res["single"], seconds_device=res["device"],
                h2d=2 * nbytes, d2h=4 * nbytes)


def time_autograd_steps(dmg, torch, w, steps, warmup, world, local, inner, profile=False, w2=None):
    """Times `steps` VI steps through the torch.autograd.Function: u = solve(q; D, mu)
    for every sample, loss = sum <w, u>, loss.backward() -> gradients w.r.t. q,
    D and mu (the transposed V-cycle plus the gradient kernel). With w2: the
    coefficients change every step (alternating between w's and w2's D, mu, as
    a sampler's iterates do), and each step first rebuilds the hierarchy in place
    (dmg_set_coefficients), inside the timed region."""
    from paper_2608_00760_b300 import autograd
    dev = torch.device("cuda", local)
    T = lambda a, g=False: torch.from_numpy(np.ascontiguousarray(a)).to(dev).requires_grad_(g)
    D, mu, q, wv = T(w["D"], True), T(w["mu"], True), T(w["q"], True), T(w["w"])
    S = dmg.Solver(D.detach(), mu.detach(), w["h"], precision=dmg.DMG_MIXED, rtol=RTOL, inner_cycles=inner,
                   autotune=AUTOTUNE[0])
    stream = torch.cuda.current_stream(dev)
    coeffs = None
    if w2 is not None:
        coeffs = [(D, mu), (T(w2["D"], True), T(w2["mu"], True))]
    count = [0]

    def step():
        Dk, muk = D, mu
        if coeffs is not None:
            Dk, muk = coeffs[count[0] % 2]
            count[0] += 1
            S.set_coefficients(Dk.detach(), muk.detach(), stream=stream)
        for x in (Dk, muk, q):
            x.grad = None
        u = autograd.DMGSolve.apply(q, Dk, muk, S, False)
        (u * wv).sum().backward()

    for _ in range(warmup):
        step()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    l0 = dmg.dmg_launch_count(S.ctx)
    barrier(world)
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    for k in range(steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    launches = dmg.dmg_launch_count(S.ctx) - l0
    prof = None
    if profile:
        prof = profiled_pass(dmg, torch, S, step, max(1, steps // 2), dmg.DMG_KERNEL_SMOOTH, True, stream, dev)
    cyc, rel = S.batch_info()
    grads_finite = all(bool(torch.isfinite(x.grad).all()) for x in (D, mu, q))
    S.close()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return dict(total_ms=max_over_ranks(world, ev[0].elapsed_time(ev[steps])), per_ms=per, launches=launches,
                prof=prof, adj_cycles=cyc, adj_rel=rel, grads_finite=grads_finite)


def run_vi(dmg, torch, args, world, local, peaks, peak_src):
    """The batched VI step: B samples x n^3, each with its own coefficients;
    per step a forward solve of every sample and the backward pass through the
    torch.autograd.Function (gradients w.r.t. q, D, mu), mixed precision; plus
    the same step for one sample at a time (a context of batch 1)."""
    from paper_2608_00760_b300 import inputs
    B, n = args.vi_batch, args.vi_size
    w = inputs.vi_batch(n, B, seed=0)
    steps = max(3, args.steps // 4)
    res = time_autograd_steps(dmg, torch, w, steps, 3, world, local, args.inner, profile=True)
    one = {k: (w[k][0] if k in ("D", "mu", "q", "w") else w[k]) for k in w}
    one["shape"] = w["shape"][1:]
    r1 = time_autograd_steps(dmg, torch, one, 3 * steps, 3, world, local, args.inner)
    w2 = inputs.vi_batch(n, B, seed=1, keys=("D", "mu"))
    rr = time_autograd_steps(dmg, torch, w, steps, 3, world, local, args.inner, w2=w2)
    del w2
    ms = res["total_ms"] / steps
    nint = B * (n - 2) ** 3
    out = dict(workload="VI step: %d tissue samples x %d^3 in one context; forward solve + backward through the "
                        "torch.autograd.Function (gradients w.r.t. q, D, mu) of every sample; rtol 1e-10; mixed "
                        "precision" % (B, n),
               value=world * B * steps / (res["total_ms"] / 1e3), unit="samples/s (fwd+VJP each)",
               ms_per_step=ms, p50_ms=percentile(res["per_ms"], 50), p99_ms=percentile(res["per_ms"], 99),
               gpu_launches_per_step=res["launches"] / steps, grads_finite=res["grads_finite"],
               adjoint_cycles_per_sample=dict(min=min(res["adj_cycles"]), max=max(res["adj_cycles"]),
                                              rel_max=max(res["adj_rel"])),
               one_at_a_time=dict(value=world * 3 * steps / (r1["total_ms"] / 1e3), unit="samples/s",
                                  ms_per_sample=r1["total_ms"] / (3 * steps),
                                  gpu_launches_per_sample=r1["launches"] / (3 * steps)),
               new_coefficients_every_step=dict(
                   value=world * B * steps / (rr["total_ms"] / 1e3), unit="samples/s",
                   ms_per_step=rr["total_ms"] / steps,
                   note="each step first rebuilds every sample's coefficient hierarchy in place "
                        "(dmg_set_coefficients, inside the timed region), alternating between two coefficient draws"))
    pr = res["prof"]
    if pr and pr["launches"]:
        dur = pr["total_ms"] / pr["launches"] / 1e3
        byt = HALF_SWEEP_BYTES_FP32 * nint
        ach = byt / dur / 1e9
        pk = peaks.get("hbm_gbs", 6400.0)
        out["roofline"] = dict(kernel="rbgs_half_sweep_fp32_level0 (all samples)", bound="hbm", achieved=ach,
                               peak=pk, unit="GB/s", frac=ach / pk,
                               frac_kernel_bytes=HALF_SWEEP_BYTES_FP32_KERNEL * nint / dur / 1e9 / pk,
                               traffic=VI_HALF_SWEEP_TRAFFIC_PER_SAMPLE_129 * B
                               if n == 129 and VI_HALF_SWEEP_TRAFFIC_PER_SAMPLE_129 else None,
                               peak_source=peak_src + " hbm_gbs", launches=pr["launches"], avg_us=dur * 1e6,
                               algorithmic_bytes=byt, bytes_per_vertex=HALF_SWEEP_BYTES_FP32)
    return out


def run_unrolled(dmg, torch, args, world, local):
    """The paper's fixed-count mode (15 FP64 V-cycles, Sec. 2.2 / 2.4) at n^3: the
    forward S_15(q), the count-matched pull-back (dmg_vjp with cycles = 15, the
    exact transpose in q) and the unrolled gradient w.r.t. q, D and mu through
    every iterate and the coarsened coefficients (dmg_vjp_unrolled, iterates
    recomputed from checkpoints)."""
    from paper_2608_00760_b300 import inputs
    n, m = args.unrolled_size, 15
    dev = torch.device("cuda", local)
    w = inputs.tissue_torch((n, n, n), 7, device=dev, keys=("D", "mu", "q", "w"))
    S = dmg.Solver(w["D"], w["mu"], 0.5, fixed_cycles=m)
    u = S.solve(w["q"])
    S.vjp(u, w["w"], cycles=m, need=(True, True, True))
    S.vjp_unrolled(w["q"], w["w"], m)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=3):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(world, e0.elapsed_time(e1) / reps)

    t_f = timed(lambda: S.solve(w["q"]))
    t_cm = timed(lambda: S.vjp(u, w["w"], cycles=m, need=(True, True, True)))
    t_u = timed(lambda: S.vjp_unrolled(w["q"], w["w"], m))
    S.close()
    return dict(workload="tissue %d^3, %d fixed FP64 V(2,2) cycles" % (n, m), forward_ms=t_f,
                count_matched_vjp_ms=t_cm, unrolled_vjp_ms=t_u, unrolled_over_forward=t_u / t_f,
                note="unrolled: forward iterates recomputed from ceil(sqrt(m)) checkpoints, states of one cycle "
                     "saved at a time; count-matched: transposed cycles plus the exact-solution coefficient "
                     "gradient")


def run_513(dmg, torch, args, world, local):
    """The larger headline size (513^3, tissue-like): fwd+VJP pairs/s mixed and FP64, and the mixed results'
    relative error against the FP64 GPU path (the oracle is too slow at this size)."""
    from paper_2608_00760_b300 import inputs
    n = args.size_513
    dev = torch.device("cuda", local)
    w = inputs.tissue_torch((n, n, n), 13, device=dev, keys=("D", "mu", "q", "w"))
    stream = torch.cuda.current_stream(dev)
    out = dict(workload="tissue-like %d^3 fwd+VJP(q,D,mu), rtol 1e-10" % n)
    res = {}
    for prec in ("mixed", "fp64"):
        S = dmg.Solver(w["D"], w["mu"], 0.5, rtol=RTOL, inner_cycles=args.inner,
                       precision=dmg.DMG_MIXED if prec == "mixed" else dmg.DMG_FP64)
        outs = [torch.empty_like(w["q"]) for _ in range(4)]
        fi, ai = dmg.dmg_info(), dmg.dmg_info()

        def step():
            st = dmg.dmg_solve_vjp(S.ctx, w["q"], w["w"], *outs, fi, ai, stream, n=S.n)
            assert st == dmg.DMG_OK, dmg.dmg_last_error(S.ctx)

        step()
        steps = 3
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        ms = max_over_ranks(world, e0.elapsed_time(e1)) / steps
        out[prec] = dict(value=world * 1e3 / ms, unit="fwd+VJP pairs/s", ms_per_step=ms, cycles=[fi.cycles, ai.cycles],
                         context_gb=dmg.dmg_device_bytes(S.ctx) / 1e9)
        res[prec] = [x.clone() for x in outs]
        S.close()
    out["mixed_vs_fp64_rel_err"] = {k: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
                                    for k, a, b in zip(("u", "qbar", "Dbar", "mubar"), res["mixed"], res["fp64"])}
    return out


def run_2d(dmg, torch, args, world, local, peaks, peak_src):
    """The 2D solver (the paper's 2D benchmarks): fwd+VJP pairs at n^2, mixed and FP64."""
    from paper_2608_00760_b300 import inputs
    n = args.size_2d
    dev = torch.device("cuda", local)
    w = inputs.tissue2d_torch((n, n), 11, device=dev)
    out = dict(workload="tissue-like %d^2 (2D, 5-point), fwd+VJP(q,D,mu), rtol 1e-10" % n)
    for prec in ("mixed", "fp64"):
        S = dmg.Solver(w["D"], w["mu"], w["h"], dim=2, rtol=RTOL, inner_cycles=args.inner,
                       precision=dmg.DMG_MIXED if prec == "mixed" else dmg.DMG_FP64)
        u = torch.empty_like(w["q"])
        qb, Db, mb = torch.empty_like(u), torch.empty_like(u), torch.empty_like(u)
        stream = torch.cuda.current_stream(dev)

        def step():   # one pair through dmg_solve_vjp, as the headline
            assert dmg.dmg_solve_vjp(S.ctx, w["q"], w["w"], u, qb, Db, mb, None, None, stream,
                                     n=S.n) == dmg.DMG_OK

        def step_seq():   # the same pair as two calls (for the kernel timing)
            assert dmg.dmg_solve(S.ctx, w["q"], u, None, stream, n=S.n) == dmg.DMG_OK
            assert dmg.dmg_vjp(S.ctx, u, w["w"], 0, qb, Db, mb, None, stream, n=S.n) == dmg.DMG_OK

        for _ in range(3):
            step()
        steps = max(3, args.steps // 2)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        barrier(world)
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for k in range(steps):
            step()
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        pr = profiled_pass(dmg, torch, S, step_seq, steps, dmg.DMG_KERNEL_SMOOTH, prec == "mixed", stream, dev)
        nl, pms = pr["launches"], pr["total_ms"]
        S.close()
        total = max_over_ranks(world, ev[0].elapsed_time(ev[steps]))
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
        r = dict(value=world * steps / (total / 1e3), unit="fwd+VJP pairs/s", ms_per_step=total / steps,
                 p50_ms=percentile(per, 50), p99_ms=percentile(per, 99))
        if nl:
            dur = pms / nl / 1e3
            if prec == "mixed":
                byt = HALF_SWEEP_BYTES_FP32 * (n - 2) ** 2
                r["roofline"] = dict(kernel="rbgs_half_sweep_2d_fp32_level0", bound="hbm", achieved=byt / dur / 1e9,
                                     peak=peaks.get("hbm_gbs", 6400.0), unit="GB/s",
                                     frac=byt / dur / 1e9 / peaks.get("hbm_gbs", 6400.0), traffic=None,
                                     peak_source=peak_src + " hbm_gbs", avg_us=dur * 1e6)
            else:
                ops = 2.5 * (n - 2) ** 2   # 4 FMA + 1 MUL per updated vertex
                r["roofline"] = dict(kernel="rbgs_half_sweep_2d_fp64_level0", bound="alu",
                                     achieved=ops / dur / 1e12, peak=FP64_OPS_PEAK[0] / 1e12, unit="TFP64-op/s",
                                     frac=ops / dur / FP64_OPS_PEAK[0], traffic=None, avg_us=dur * 1e6,
                                     peak_source="dmg_probe_fma, measured in this run")
        out[prec] = r
    return out


def run_levels(dmg, torch, S, w, local):
    """Where a pair's time goes: for each kernel kind and level of the headline
    context, the launches per pair and their event-timed duration (dmg_profile;
    runs of consecutive half-sweeps share one event pair), from the two-call
    form of the pair so that no second lane runs beside the kernel."""
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    q, wv = T(w["q"]), T(w["w"])
    u = torch.empty_like(q)
    qb, Db, mb = torch.empty_like(q), torch.empty_like(q), torch.empty_like(q)

    def step():
        assert dmg.dmg_solve(S.ctx, q, u, None, stream, n=S.n) == dmg.DMG_OK
        assert dmg.dmg_vjp(S.ctx, u, wv, 0, qb, Db, mb, None, stream, n=S.n) == dmg.DMG_OK

    names = [(dmg.DMG_KERNEL_SMOOTH, "smooth"), (dmg.DMG_KERNEL_RESTRICT, "restrict"),
             (dmg.DMG_KERNEL_PROLONG, "prolong"), (dmg.DMG_KERNEL_TAIL, "tail"),
             (dmg.DMG_KERNEL_RESIDUAL, "residual_fp64"), (dmg.DMG_KERNEL_GRAD, "grad")]
    reps = 3
    rows, total = {}, 0.0
    for lev in range(dmg.dmg_levels(S.ctx)):
        for fp32 in (True, False):
            for kind, name in names:
                dmg.dmg_profile_begin(S.ctx, kind, lev, fp32, max_launches=4096)
                for _ in range(reps):
                    step()
                torch.cuda.synchronize(dev)
                _, n, ms = dmg.dmg_profile_end(S.ctx)
                if n:
                    key = "L%d %s %s" % (lev, "fp32" if fp32 else "fp64", name)
                    rows[key] = dict(launches_per_pair=n / reps, avg_us=1e3 * ms / n, us_per_pair=1e3 * ms / reps)
                    total += 1e3 * ms / reps
    return dict(note="event-timed inside the replayed graphs (a few us of event-node cost per run of launches "
                     "included); two-call pair", kernels=rows, sum_us_per_pair=total)


def run_setup(dmg, torch, args, world, local):
    """The cost of row a1 (the coefficient hierarchy): dmg_setup (allocation, hierarchy, coarsest inverse, no
    autotuning), dmg_set_coefficients (the hierarchy rebuilt in place for new coefficients) and dmg_slot_load (one
    slot of a serving pool), wall-clock around each synchronous call, median of 3 (setup) or 5 (rebuilds)."""
    from paper_2608_00760_b300 import inputs
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    out = dict(note="milliseconds per call; setup includes every cudaMalloc of the context")

    def med(fn, reps):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize(dev)
            ts.append(1e3 * (time.perf_counter() - t0))
        return float(np.median(ts))

    sizes = [(257, "mixed"), (257, "fp64")] + ([(args.size_513, "mixed")] if args.size_513 > 0 else [])
    for n, prec in sizes:
        w = inputs.tissue_torch((n, n, n), 21, device=dev, keys=("D", "mu"))
        p = dmg.DMG_MIXED if prec == "mixed" else dmg.DMG_FP64
        holder = []

        def setup():
            holder.append(dmg.Solver(w["D"], w["mu"], 0.5, precision=p, autotune=0))

        t_setup = med(setup, 3)
        S = holder[-1]
        for x in holder[:-1]:
            x.close()
        t_set = med(lambda: S.set_coefficients(w["D"], w["mu"], stream=stream), 5)
        out["%d^3_%s" % (n, prec)] = dict(dmg_setup_ms=t_setup, dmg_set_coefficients_ms=t_set,
                                          context_gb=dmg.dmg_device_bytes(S.ctx) / 1e9)
        S.close()
        del w
    for n in (129, 257):
        w = inputs.tissue_torch((n, n, n), 22, device=dev, keys=("D", "mu"))
        prm = dmg.dmg_default_params(nx=n, ny=n, nz=n, h=0.5, batch=4, precision=dmg.DMG_MIXED)
        ones = torch.ones((4, n, n, n), dtype=torch.float64, device=dev)
        st, ctx = dmg.dmg_setup(prm, ones, ones, stream=stream)
        del ones
        assert st == dmg.DMG_OK, dmg.dmg_last_error(None)
        nn = n ** 3
        t_load = med(lambda: dmg.dmg_slot_load(ctx, 1, w["D"], w["mu"], stream, n=nn), 5)
        out["slot_load_%d^3_mixed_ms" % n] = t_load
        dmg.dmg_destroy(ctx)
        del w
    return out


SERVE_SHAPES = [(33, 33, 33), (65, 65, 65), (129, 129, 129), (257, 257, 257), (129, 257, 257)]


def serve_stream(dmg, torch, args, world, rank, local, rate, nreq, pyramid=False):
    """One served stream of nreq Poisson arrivals at `rate` per second (mixed precision, rtol 1e-10)."""
    from paper_2608_00760_b300 import serve
    dev = torch.device("cuda", local)
    reqs = serve.poisson_stream(nreq, rate, SERVE_SHAPES, seed=1000 + rank)
    server = serve.Server(SERVE_SHAPES, budget_bytes=args.serve_budget_gb * 1e9, device=dev,
                          params=dict(precision=dmg.DMG_MIXED, rtol=RTOL, inner_cycles=args.inner),
                          pyramid=pyramid)
    try:
        warm = serve.poisson_stream(3 * len(SERVE_SHAPES), 1e4, SERVE_SHAPES, seed=99)
        server.run(warm, realtime=False, keep_outputs=False)      # graph capture, outside the measurement
        barrier(world)
        served, st = server.run(reqs, keep_outputs=False)
        slots = {"x".join(map(str, s[::-1])): server.slots[s] for s in server.pools}
        pyramids = ["+".join("x".join(map(str, s[::-1])) for s in p.chain) for p in server.unique_pools()
                    if len(p.chain) > 1]
        pool_gb = server.pool_bytes / 1e9
    finally:
        server.close()
    return reqs, served, st, dict(slots=slots, pyramid_pools=pyramids), pool_gb


def run_serving(dmg, torch, args, world, rank, local):
    """The request stream: Poisson arrivals of forward, JVP and VJP requests
    (1:1:2) on grids drawn uniformly from SERVE_SHAPES, tissue coefficients with
    per-request seeds, served with continuous batching under the memory budget
    (mixed precision, rtol 1e-10); then the same requests one at a time in FP64."""
    from paper_2608_00760_b300 import serve
    dev = torch.device("cuda", local)
    reqs, served, st, layout, pool_gb = serve_stream(dmg, torch, args, world, rank, local, args.serve_rate,
                                                      args.serve_requests)
    secs = max_over_ranks(world, st["seconds"])
    pyr = None
    if args.serve_pyramid:
        preqs, _, pst, playout, _ = serve_stream(dmg, torch, args, world, rank, local, args.serve_rate,
                                                 args.serve_requests, pyramid=True)
        psecs = max_over_ranks(world, pst["seconds"])
        pyr = dict(rate=args.serve_rate, value=world * sum(r.solves for r in preqs) / psecs
                   if pst["ok"] == len(preqs) else None, unit="solves/s", requests_per_s=world * pst["ok"] / psecs,
                   p50_ms=pst["p50_ms"], p99_ms=pst["p99_ms"], seconds=psecs, pyramid_pools=playout["pyramid_pools"],
                   note="the cube shapes in one pyramid pool: one launch per kernel and level for every slot of "
                        "every shape holding that level")
    low = None
    if args.serve_rate_low > 0:
        lreqs, lserved, lst, _, _ = serve_stream(dmg, torch, args, world, rank, local, args.serve_rate_low,
                                                 args.serve_requests)
        lsecs = max_over_ranks(world, lst["seconds"])
        low = dict(rate=args.serve_rate_low, value=world * sum(r.solves for r in lreqs) / lsecs
                   if lst["ok"] == len(lreqs) else None, unit="solves/s", requests_per_s=world * lst["ok"] / lsecs,
                   ok=lst["ok"], requests=len(lreqs), p50_ms=lst["p50_ms"], p99_ms=lst["p99_ms"], seconds=lsecs)
    t_alone = serve.run_one_at_a_time(reqs, params=dict(precision=dmg.DMG_FP64, rtol=RTOL), device=dev)
    t_alone = max_over_ranks(world, t_alone)
    nsolves = sum(r.solves for r in reqs)
    cyc = [c for r in served for c in r.cycles]
    return dict(workload="%d Poisson arrivals at %g/s; shapes %s (x*y*z) uniform; fwd:JVP:VJP = 1:1:2; tissue "
                         "coefficients with per-request seeds; %g GB budget; mixed precision, rtol 1e-10"
                         % (len(reqs), args.serve_rate, ", ".join("x".join(map(str, s[::-1])) for s in SERVE_SHAPES),
                            args.serve_budget_gb),
                value=world * nsolves / secs if st["ok"] == len(reqs) else None, unit="solves/s",
                requests_per_s=world * st["ok"] / secs, ok=st["ok"], requests=len(reqs),
                p50_ms=st["p50_ms"], p99_ms=st["p99_ms"], seconds=secs,
                slots=layout["slots"], pyramid_pools=layout["pyramid_pools"], pools_gb=pool_gb,
                cycles_mean=float(np.mean(cyc)) if cyc else None,
                lower_rate=low, pyramid_variant=pyr,
                one_at_a_time_fp64=dict(value=world * nsolves / t_alone, unit="solves/s",
                                        requests_per_s=world * len(reqs) / t_alone, seconds=t_alone,
                                        api="dmg_setup + dmg_solve/dmg_jvp/dmg_vjp per request, batch 1"))


def _oracle_sample_times(w):
    """Times of the FP64 CPU oracle (single-threaded C) on one bounded sample of
    a workload: one forward V-cycle, one residual norm, one transposed V-cycle
    and one coefficient-gradient evaluation, at the full grid."""
    import oracle
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    z = np.zeros(w["shape"])
    t0 = time.perf_counter()
    u1 = H.vcycle(w["q"], z)
    t1 = time.perf_counter()
    H.rel_residual(w["q"], u1)
    t2 = time.perf_counter()
    l1 = H.vcycle(w["w"], z, transposed=True)
    t3 = time.perf_counter()
    oracle.grad(w["D"], w["h"], u1, l1)
    t4 = time.perf_counter()
    return dict(fwd=t1 - t0, res=t2 - t1, adj=t3 - t2, grad=t4 - t3, total=t4 - t0)


def _pair_seconds(t, m_fwd, m_adj):
    """One fwd+VJP pair: m_fwd forward cycles and m_adj transposed cycles, each
    followed by a residual norm, plus one gradient evaluation."""
    return m_fwd * (t["fwd"] + t["res"]) + m_adj * (t["adj"] + t["res"]) + t["grad"]


def _oracle_worker(path, h):
    """One process of the all-core run: the bounded sample on the arrays saved at path."""
    w = {k: np.load(os.path.join(path, k + ".npy"), mmap_mode="r") for k in ("D", "mu", "q", "w")}
    w = {k: np.ascontiguousarray(v) for k, v in w.items()}
    w["h"], w["shape"] = h, w["D"].shape
    return _oracle_sample_times(w)


def _all_core_processes(shape):
    """Concurrent oracle processes for the all-core run: one per usable core,
    as many as host memory holds (about 1.6 GB per process at 257^3)."""
    cores = host_info()["usable"] or 1
    per = 1.6e9 * float(np.prod(shape)) / 257 ** 3
    avail = 8e9
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    avail = 1024.0 * float(line.split()[1])
                    break
    except Exception:
        pass
    return max(1, min(cores, int(0.6 * avail // per), 128))


def cpu_baseline_leg(dmg, torch, w, m_fwd, m_adj, local, inner):
    """The FP64 CPU oracle as it stands, on this host's cores (the reported CPU
    baseline), plus the oracle's own check of the GPU path at 65^3.

    * single thread: the bounded sample (one forward and one transposed
      V-cycle, one residual norm, one gradient evaluation) at the full grid,
      scaled to a fwd+VJP pair with the GPU run's cycle counts;
    * all cores: the same sample in one process per usable core at once (the
      oracle is single-threaded C; independent pairs are how a sampler would
      use the host), throughput = sum of the processes' pair rates;
    * the scaling is checked against a measured full pair of the oracle at
      65^3 (predicted from the same per-cycle sample there);
    * 65^3 parity (the tissue recipe's errors the configuration asks for):
      the GPU's mixed and FP64 fwd+VJP results against the oracle's, relative
      L2 and max-entry errors of u, qbar, Dbar, mubar."""
    import multiprocessing as mp

    import oracle
    from paper_2608_00760_b300 import inputs
    oracle.build()
    host = host_info()
    # single thread, full grid
    t = _oracle_sample_times(w)
    pair1 = _pair_seconds(t, m_fwd, m_adj)
    # all cores, full grid
    nproc = _all_core_processes(w["shape"])
    with tempfile.TemporaryDirectory() as d:
        for k in ("D", "mu", "q", "w"):
            np.save(os.path.join(d, k + ".npy"), w[k])
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(nproc) as pool:
            ts = pool.starmap(_oracle_worker, [(d, w["h"])] * nproc)
        wall = time.perf_counter() - t0
    rate_all = sum(1.0 / _pair_seconds(x, m_fwd, m_adj) for x in ts)
    # 65^3: measured oracle pair, predicted pair, and the GPU's errors against it
    s = inputs.tissue(65, seed=3)
    H = oracle.Hierarchy(s["D"], s["mu"], s["h"])
    t0 = time.perf_counter()
    ur, mf, _ = H.solve(s["q"], rtol=RTOL)
    qr, Dr, mr, ma = H.vjp(ur, s["w"], rtol=RTOL)
    meas65 = time.perf_counter() - t0
    pred65 = _pair_seconds(_oracle_sample_times(s), mf, ma)
    dev = torch.device("cuda", local)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    errs = {}
    for prec in ("mixed", "fp64"):
        S = dmg.Solver(T(s["D"]), T(s["mu"]), s["h"], rtol=RTOL, inner_cycles=inner,
                       precision=dmg.DMG_MIXED if prec == "mixed" else dmg.DMG_FP64)
        u = S.solve(T(s["q"]))
        qb, Db, mb = S.vjp(u, T(s["w"]))
        S.close()
        e = {}
        for k, a, b in (("u", u, ur), ("qbar", qb, qr), ("Dbar", Db, Dr), ("mubar", mb, mr)):
            a = a.cpu().numpy()
            e[k] = dict(rel_l2=float(np.linalg.norm(a - b) / np.linalg.norm(b)),
                        rel_max=float(np.max(np.abs(a - b)) / np.max(np.abs(b))))
        errs[prec] = e
    shape = "x".join(map(str, w["shape"]))
    return dict(value=1.0 / pair1, unit=UNIT, cores=1, kind="oracle",
                sample="1 forward + 1 transposed V(2,2) cycle, 1 residual norm and 1 gradient evaluation of the FP64 "
                       "oracle at %s (%.1f s), scaled to %d + %d cycles per fwd+VJP pair" %
                       (shape, t["total"], m_fwd, m_adj),
                host=host,
                all_cores=dict(value=rate_all, unit=UNIT, cores=nproc, processes=nproc, wall_s=wall,
                               sample="the same sample in %d concurrent single-threaded oracle processes; value = "
                                      "sum of their pair rates" % nproc),
                scaling_check_65=dict(measured_pair_s=meas65, predicted_pair_s=pred65, cycles=[mf, ma],
                                      ratio=pred65 / meas65),
                oracle_parity_65=dict(workload="tissue-like 65^3 (seed 3), fwd+VJP(q,D,mu), rtol 1e-10 on both "
                                               "sides", **errs))


def reference_arm(args, rank):
    """The oracle as it stands, on this host's cores, on the same workload: every
    step is one forward V-cycle plus its residual norm at the full grid (about
    5 s single-threaded); one transposed cycle and one gradient evaluation are
    timed once, and the pair time is m_fwd forward cycles + m_adj transposed
    cycles + one gradient, with the cycle counts the oracle itself needs on the
    same recipe at 129^3 (the V-cycle's contraction is h-independent)."""
    if rank != 0:
        return
    import oracle
    from paper_2608_00760_b300 import inputs
    oracle.build()
    small = inputs.tissue(129, seed=0)
    Hs = oracle.Hierarchy(small["D"], small["mu"], small["h"])
    _, m_fwd, _ = Hs.solve(small["q"], rtol=RTOL)
    _, m_adj, _ = Hs.adjoint(small["w"], rtol=RTOL)
    w = make_inputs(args.size)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    z = np.zeros(w["shape"])

    def fwd_cycle():
        t0 = time.perf_counter()
        u1 = H.vcycle(w["q"], z)
        H.rel_residual(w["q"], u1)
        return time.perf_counter() - t0, u1

    for _ in range(args.warmup):
        fwd_cycle()
    times = []
    for _ in range(args.steps):
        t, u1 = fwd_cycle()
        times.append(t)
    t0 = time.perf_counter()
    l1 = H.vcycle(w["w"], z, transposed=True)
    H.rel_residual(w["w"], l1)
    t_adj = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.grad(w["D"], w["h"], u1, l1)
    t_grad = time.perf_counter() - t0
    t_fwd = float(np.mean(times))
    t_pair = m_fwd * t_fwd + m_adj * t_adj + t_grad
    v = 1.0 / t_pair
    sample = ("each step: 1 forward V(2,2) cycle + residual norm of the FP64 oracle at %d^3 (mean %.2f s); "
              "pair = %d forward cycles + %d transposed cycles (%.2f s each, timed once) + 1 gradient (%.2f s); "
              "cycle counts from the oracle's own 129^3 solves" % (args.size, t_fwd, m_fwd, m_adj, t_adj, t_grad))
    # ms_per_step is the measured time of one timed step (one forward cycle and
    # its residual norm); the pair time the value comes from is ms_per_pair
    out = dict(metric=METRIC, value=v, unit=UNIT, impl="reference", n_gpus=args.gpus, steps=args.steps,
               warmup=args.warmup, ms_per_step=1e3 * t_fwd, ms_per_pair=1e3 * t_pair, higher_is_better=True,
               scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
               config=dict(workload="tissue-like %d^3 fwd+VJP(q,D,mu), rtol 1e-10" % args.size,
                           grid=[args.size] * 3, h_mm=0.5, rtol=RTOL, precision="fp64 (CPU oracle, single thread)"),
               cpu_baseline=dict(value=v, unit=UNIT, cores=1, kind="oracle", sample=sample, host=host_info()),
               e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="dmg", choices=["dmg", "reference"])
    ap.add_argument("--size", type=int, default=N_SIDE)
    ap.add_argument("--only", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--inner", type=int, default=3, help="FP32 V-cycles per FP64 refinement step (mixed)")
    ap.add_argument("--vi-batch", type=int, default=64, help="samples of the batched VI step (0: skip it)")
    ap.add_argument("--vi-size", type=int, default=129)
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests of the serving stream (0: skip it)")
    ap.add_argument("--unrolled-size", type=int, default=257, help="grid of the unrolled-gradient timing (0: skip)")
    ap.add_argument("--vi-only", action="store_true", help="run only the batched VI step and print its object")
    ap.add_argument("--size-2d", type=int, default=4097, help="grid of the 2D solver timing (0: skip)")
    ap.add_argument("--size-513", type=int, default=513, help="larger 3D grid timed next to the headline (0: skip)")
    ap.add_argument("--autotune", type=int, default=1, help="tile autotuner at setup (dmg_params.autotune)")
    ap.add_argument("--twin", type=int, default=1,
                    help="dmg_params.twin_adjoint of the headline contexts: 1 runs the adjoint solve of a pair "
                         "beside the forward one")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-budget-gb", type=float, default=80.0)
    ap.add_argument("--serve-rate-low", type=float, default=60.0,
                    help="arrival rate of a second stream below capacity (0: skip it)")
    ap.add_argument("--no-setup", action="store_true", help="skip the setup-cost timings")
    ap.add_argument("--no-levels", action="store_true", help="skip the per-level kernel timings")
    ap.add_argument("--serve-pyramid", type=int, default=1,
                    help="also serve the stream with the cube shapes in one pyramid pool (0: skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args, int(os.environ.get("RANK", "0")))
        return
    args.warmup = max(args.warmup, 3)
    AUTOTUNE[0] = args.autotune
    TWIN[0] = args.twin
    world, rank, local = dist_setup()

    import torch
    from paper_2608_00760_b300 import dmg
    dmg.lib()
    torch.cuda.set_device(local)
    st, FP64_OPS_PEAK[0] = dmg.dmg_probe_fma(True)
    st32, fp32_rate = dmg.dmg_probe_fma(False)
    if st != dmg.DMG_OK or not FP64_OPS_PEAK[0] > 0:
        raise RuntimeError("dmg_probe_fma failed: %s" % dmg.dmg_strerror(st))
    if args.vi_only:
        peaks, peak_src = load_peaks()
        vi = run_vi(dmg, torch, args, world, local, peaks, peak_src)
        if rank == 0:
            print(json.dumps(vi))
        return
    w = make_inputs(args.size)
    npts = int(np.prod(w["shape"]))
    nint = int(np.prod([s - 2 for s in w["shape"]]))
    peaks, peak_src = load_peaks()

    results = {}
    precisions = {"both": ["mixed", "fp64"], "mixed": ["mixed"], "fp64": ["fp64"]}[args.only]
    for prec in precisions:
        p = dmg.DMG_MIXED if prec == "mixed" else dmg.DMG_FP64
        prof = (dmg.DMG_KERNEL_SMOOTH, prec == "mixed")
        results[prec] = run_arm(dmg, torch, w, p, args.steps, args.warmup, world, local, profile=prof,
                                clocks=(prec == precisions[0]), inner=args.inner if prec == "mixed" else 1)

    head = results[precisions[0]]
    S = head["solver"]
    tiles = {"fp32" if prec == "mixed" else "fp64": ["%dx%d" % t for t in results[prec]["solver"].tiles(prec == "mixed")]
             for prec in precisions}
    ms = head["total_ms"] / args.steps
    value = job_throughput(world, args.steps, head["total_ms"])

    def roofline(res, prec):
        pr = res["prof"]
        if not pr or not pr["launches"]:
            return None
        dur = pr["total_ms"] / pr["launches"] / 1e3
        if prec == "mixed":
            byt = HALF_SWEEP_BYTES_FP32 * nint
            ach = byt / dur / 1e9
            pk = peaks.get("hbm_gbs", 6400.0)
            return dict(kernel="rbgs_half_sweep_fp32_level0", bound="hbm", achieved=ach, peak=pk, unit="GB/s",
                        frac=ach / pk, frac_kernel_bytes=HALF_SWEEP_BYTES_FP32_KERNEL * nint / dur / 1e9 / pk,
                        traffic=HALF_SWEEP_TRAFFIC["fp32"] if args.size == 257 else None,
                        peak_source=peak_src + " hbm_gbs", launches=pr["launches"], avg_us=dur * 1e6,
                        algorithmic_bytes=byt, bytes_per_vertex=HALF_SWEEP_BYTES_FP32,
                        timing="CUDA event nodes around each run of consecutive launches of the kernel (the "
                               "half-sweeps of one smoothing step) inside the replayed graphs, divided by the "
                               "launches in the run, in a second pass of the same pairs after the timed one "
                               "(%.2f ms per pair with the event nodes)" % pr["pass_ms_per_step"],
                        note="algorithmic bytes: 20 B per interior vertex per full FP32 sweep (read u, f, D, mu; "
                             "write u), 10 B per half-sweep; frac_kernel_bytes charges the 12 B the colour kernel "
                             "moves")
        ops = HALF_SWEEP_FP64_OPS * nint
        ach = ops / dur / 1e12
        return dict(kernel="rbgs_half_sweep_fp64_level0", bound="alu", achieved=ach, peak=FP64_OPS_PEAK[0] / 1e12,
                    unit="TFP64-op/s", frac=ach / (FP64_OPS_PEAK[0] / 1e12),
                    traffic=HALF_SWEEP_TRAFFIC["fp64"] if args.size == 257 else None,
                    peak_source="dmg_probe_fma FP64 FMA rate, measured in this run", launches=pr["launches"],
                    avg_us=dur * 1e6, algorithmic_fp64_ops=ops,
                    timing="CUDA event nodes around each run of consecutive launches, second pass (%.2f ms per "
                           "pair with the event nodes)" % pr["pass_ms_per_step"])

    def gbs(res, prec):
        # algorithmic HBM bytes of one pair divided by its time (see the design notes for the per-cycle bytes)
        per_cycle = 272.0 if prec == "fp64" else 136.0
        outer = 56.0 if prec == "mixed" else 0.0
        cyc = res["fwd_cycles"] + res["adj_cycles"]
        byt = npts * (per_cycle * cyc + outer * (res["fwd_outer"] + res["adj_outer"]) + 40.0)
        return byt / (res["total_ms"] / args.steps / 1e3) / 1e9

    out = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
               ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None,
               dtype="f32-inner/f64-outer" if precisions[0] == "mixed" else "f64", data="synthetic",
               config=dict(workload="tissue-like %d^3 fwd+VJP(q,D,mu), rtol 1e-10" % args.size,
                           grid=list(w["shape"]), h_mm=w["h"], rtol=RTOL, precision=precisions[0],
                           parallelism="replicas" if world > 1 else "single-gpu",
                           inner_cycles=args.inner if precisions[0] == "mixed" else None,
                           l2="inputs larger than L2 (each FP64 field %.0f MB > 126 MB); no flush" % (8 * npts / 1e6),
                           setup="dmg_setup once per coefficient field, outside the timed region",
                           autotune=args.autotune, tiles_per_level=tiles),
               p50_ms=percentile(head["per_ms"], 50), p99_ms=percentile(head["per_ms"], 99),
               hbm_gbs_algorithmic=gbs(head, precisions[0]),
               cycles=dict(fwd=head["fwd_cycles"], adj=head["adj_cycles"], fwd_outer=head["fwd_outer"],
                           adj_outer=head["adj_outer"], fwd_rel=head["fwd_rel"], adj_rel=head["adj_rel"]),
               gpu_launches=head["launches"], gpu_launches_per_step=head["launches"] / args.steps,
               device_memory_gb=dict(context=dmg.dmg_device_bytes(S.ctx) / 1e9,
                                     note="the context and its twin (the adjoint lane dmg_solve_vjp creates on "
                                          "its first call, outside the timed region); nothing is allocated "
                                          "inside a pair"),
               pair_api="dmg_solve_vjp: the adjoint solve (it needs only w) runs in the twin context on its own "
                        "stream and host thread while the forward one runs; results bit for bit those of "
                        "dmg_solve + dmg_vjp",
               sequential_ms_per_step=head["seq_ms"],
               roofline=roofline(head, precisions[0]), clocks=head["clocks"],
               measured_rates=dict(fp64_fma_per_s=FP64_OPS_PEAK[0], fp32_fma_per_s=fp32_rate,
                                   source="dmg_probe_fma (independent FMA chains on every SM, CUDA events)"))
    for prec in precisions[1:]:
        r = results[prec]
        out[prec] = dict(value=job_throughput(world, args.steps, r["total_ms"]), unit=UNIT,
                         ms_per_step=r["total_ms"] / args.steps, p50_ms=percentile(r["per_ms"], 50),
                         p99_ms=percentile(r["per_ms"], 99), hbm_gbs_algorithmic=gbs(r, prec),
                         cycles=dict(fwd=r["fwd_cycles"], adj=r["adj_cycles"]), gpu_launches=r["launches"],
                         roofline=roofline(r, prec))
    if "mixed" in results and "fp64" in results:
        a, b = results["mixed"]["out"], results["fp64"]["out"]
        out["mixed_vs_fp64_rel_err"] = {k: float(torch.linalg.norm(x - y) / torch.linalg.norm(y))
                                        for k, x, y in zip(("u", "qbar", "Dbar", "mubar"), a, b)}
    out["levels"] = (run_levels(dmg, torch, head["solver"], w, local)
                     if rank == 0 and world == 1 and not args.no_levels else None)
    for r in results.values():
        r["solver"].close()
        r.pop("out", None)

    if not args.no_e2e:
        ns = max(6, args.steps)
        e = run_e2e(dmg, torch, w, dmg.DMG_MIXED if precisions[0] == "mixed" else dmg.DMG_FP64,
                    ns, 1, world, local, inner=args.inner)
        out["e2e"] = dict(value=world * ns / e["seconds"], unit=UNIT, h2d_bytes_per_step=e["h2d"],
                          d2h_bytes_per_step=e["d2h"], steps=ns,
                          api="dmg_solve_vjp_many over %d pairs with pinned host buffers (q, w in; u, qbar, Dbar, "
                              "mubar out per pair; transfers overlapped with the neighbouring pairs' solves)" % ns,
                          single_call=dict(value=world * ns / e["seconds_single"], unit=UNIT,
                                           api="dmg_solve_vjp, one call per pair"))
        out["stream_of_pairs_device"] = dict(
            value=world * ns / e["seconds_device"], unit=UNIT, steps=ns,
            api="dmg_solve_vjp_many over %d pairs, inputs and outputs resident on the device (host clock around the "
                "call): each pair's gradient and read-out overlap the next pair's solves" % ns)
    else:
        out["e2e"] = None
        out["stream_of_pairs_device"] = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        m_f = results.get("fp64", head)["fwd_cycles"]
        m_a = results.get("fp64", head)["adj_cycles"]
        out["cpu_baseline"] = cpu_baseline_leg(dmg, torch, w, m_f, m_a, local, args.inner)
    else:
        out["cpu_baseline"] = None
    out["vi_batch"] = run_vi(dmg, torch, args, world, local, peaks, peak_src) if args.vi_batch > 0 else None
    out["serving"] = (run_serving(dmg, torch, args, world, rank, local) if args.serve_requests > 0 else None)
    out["unrolled"] = run_unrolled(dmg, torch, args, world, local) if args.unrolled_size > 0 else None
    out["setup"] = run_setup(dmg, torch, args, world, local) if not args.no_setup else None
    out["two_d"] = run_2d(dmg, torch, args, world, local, peaks, peak_src) if args.size_2d > 0 else None
    out["c3_large"] = run_513(dmg, torch, args, world, local) if args.size_513 > 0 else None
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
