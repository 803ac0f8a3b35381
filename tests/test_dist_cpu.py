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
