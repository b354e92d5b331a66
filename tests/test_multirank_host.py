"""The multi-replica aggregation of bench.py (sum of work, max of time over ranks) on two
gloo ranks on the CPU.  The single-cell path has no exchange step: ranks are independent
replicas and only these two reductions cross ranks."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = 1000.0 * (rank + 1)
    seconds = 0.5 + rank
    tot, mx = bench.aggregate_over_ranks(units, seconds, world, device="cpu")
    out.put((rank, tot, mx))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tot, mx in res:
        assert tot == 3000.0      # whole-job units: sum over ranks
        assert mx == 1.5          # timed region: slowest rank


def test_aggregate_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(7.0, 2.0, 1) == (7.0, 2.0)
