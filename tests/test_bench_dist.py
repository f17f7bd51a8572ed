"""bench.py's multi-rank helpers on CPU: two gloo ranks agree on the slowest
rank's time, and the whole-job value counts every rank's queries (replicas,
weak scaling, no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import bench

    bench.init_dist(world)                     # gloo here: no CUDA device
    assert dist.get_world_size() == world and dist.get_rank() == rank
    assert bench.dist_env() == (rank, rank, world)
    slow = bench.reduce_max(1.0 + rank, world)       # rank 1 is the slow one
    bench.barrier(world)
    choice = bench.broadcast_ints([2 + rank, 48 - rank], world)   # rank 0's operating point
    out[rank] = (slow, bench.aggregate_value(10_000, world, slow), tuple(choice))
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    ctx = torch.multiprocessing.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 10_000.0, (2, 48))


def test_single_process_helpers():
    import bench

    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.broadcast_ints([3, 40], 1) == [3, 40]
    assert bench.aggregate_value(500, 1, 0.25) == 2000.0
