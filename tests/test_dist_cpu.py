"""bench.py's multi-rank plumbing on CPU with world_size-2 gloo ranks: the
barrier, the max-over-ranks of the timed region and the whole-job throughput
(a single solve does not shard; N ranks run N replicas)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    t = bench.max_over_ranks(w, 100.0 + 50.0 * rank)   # rank 1 is the slow one
    v = bench.job_throughput(w, 10, t)
    with open(os.path.join(outdir, "rank%d.txt" % rank), "w") as fh:
        fh.write("%r %r\n" % (t, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    vals = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(2)]
    for t, v in vals:
        assert float(t) == 150.0
        assert float(v) == pytest.approx(2 * 10 / 0.150)


def test_single_rank_defaults():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1, 3.5) == 3.5
    assert bench.job_throughput(1, 20, 1000.0) == pytest.approx(20.0)


def test_reference_arm_prints_one_complete_line():
    # the oracle arm on a small grid: one JSON line with the contract's keys,
    # the timed steps' own duration as ms_per_step, and host-only e2e bytes
    import json
    import subprocess
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--size", "33", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["ms_per_step"] < d["ms_per_pair"] and abs(d["value"] - 1e3 / d["ms_per_pair"]) <= 1e-9 * d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--size", "33", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "{" not in r.stdout
