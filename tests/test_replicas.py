"""Multi-GPU runs are independent replicas (the path's only cross-rank step is
the timing reduction).  Check that aggregation on CPU ranks (gloo, world 2):
the job time is the slowest rank's and the value counts every replica."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total, value = bench.aggregate(100.0 * (rank + 1), 17424, world)
    q.put((rank, total, value))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for _, total, value in out:
        assert total == 200.0
        assert value == pytest.approx(2 * 17424 / 0.2)
