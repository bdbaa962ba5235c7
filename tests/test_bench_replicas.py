"""Replica aggregation of bench.py across ranks (torch.distributed, gloo,
world size 2, on CPU): the whole-job value is the units of all ranks over
the slowest rank's time, identical on every rank."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank              # rank 1 is the slower one
    value, ms_max = bench.replica_value(4.0, ms, world, dist, device="cpu")
    out.put((rank, value, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_value():
    mp = pytest.importorskip("torch.multiprocessing")
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
    for rank, value, ms_max in res:
        assert ms_max == 150.0
        assert abs(value - 4.0 * 2 / 0.150) < 1e-9


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.replica_value(3.0, 200.0, 1, None)
    assert ms == 200.0 and abs(value - 15.0) < 1e-12
