"""bench.py's host logic on CPU: two gloo ranks agree on the slowest rank's
time and on rank 0's operating point, the whole-job value counts every
rank's queries (replicas, weak scaling, no collective on the data path), and
the operating-point choice follows its rule."""
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


def test_operating_point_choice():
    import bench

    def c(width, ef, rmin, ms):
        return {"width": width, "ef": ef, "recall_at_10_min_p_bin": rmin, "ms": ms}

    cal = [c(1, 48, 0.952, 1.85), c(2, 48, 0.953, 1.596), c(3, 48, 0.951, 1.585)]
    assert bench.choose_operating_point(cal, 0.95)["width"] == 2      # 3 is within 1 %
    cal[2]["ms"] = 1.40
    assert bench.choose_operating_point(cal, 0.95)["width"] == 3      # clearly faster
    cal[2]["recall_at_10_min_p_bin"] = 0.94
    assert bench.choose_operating_point(cal, 0.95)["width"] == 2      # misses the target
    low = [c(1, 512, 0.61, 9.0), c(2, 512, 0.62, 8.0)]
    assert bench.choose_operating_point(low, 0.95)["width"] == 2      # none meets it
    assert bench.choose_operating_point([c(1, 48, 0.97, None)], 0.95)["ef"] == 48


def test_recall_per_bin_on_the_p_grid():
    """Every grid value 0.5, 0.6, ..., 2.0 (as FP32) lands in its own bin, and
    a bin's recall is the mean of its queries' |found & true| / k."""
    import numpy as np

    import bench
    from paper_2605_02030_gb300 import inputs as I

    p = np.repeat(np.array([0.5 + 0.1 * i for i in range(16)], np.float32), 2)
    gt = np.tile(np.arange(10), (len(p), 1))
    ids = gt.copy()
    ids[0, :3] = [-1, 97, 98]          # query 0 (p = 0.5) finds 7 of 10
    ids[31, 9] = 99                    # query 31 (p = 2.0) finds 9 of 10
    bins = I.p_bin_of(I.WORKLOADS["sift1m"], p)
    assert (bins == np.repeat(np.arange(16), 2)).all()
    overall, per = bench.recall_per_bin(ids, gt, bins, 10)
    assert sorted(per) == list(range(16))
    assert per[0] == (0.7 + 1.0) / 2 and per[15] == (1.0 + 0.9) / 2
    assert all(per[b] == 1.0 for b in range(1, 15))
    assert abs(overall - (32 - 0.3 - 0.1) / 32) < 1e-12


def test_uniform_p_bins():
    """p ~ U(0.5, 2] falls into 16 equal bins (lo + b h, lo + (b + 1) h],
    h = 1.5 / 16: each edge belongs to the bin below it."""
    import numpy as np

    from paper_2605_02030_gb300 import inputs as I

    w = I.WORKLOADS["sift1m_fp16"]
    h = 1.5 / 16
    edges = 0.5 + h * np.arange(1, 17)
    assert np.allclose(I.p_bin_of(w, edges), np.arange(16))
    assert np.allclose(I.p_bin_of(w, edges - h / 2), np.arange(16))
    assert (I.p_bin_of(w, edges[:-1] + 1e-6) == np.arange(1, 16)).all()
    p, _, _ = I.query_params(w)
    counts = np.bincount(I.p_bin_of(w, p), minlength=16)
    assert counts.sum() == w.nq and counts.min() > 0.8 * w.nq / 16


def test_calibration_set_is_held_out():
    """The calibration queries come from streams of their own: same recipe
    (shape, value range), different draws."""
    import numpy as np

    from paper_2605_02030_gb300 import inputs as I

    w = I.WORKLOADS["sift1m_fp16"].scaled(n=2000, nq=500)
    q = I.query_vectors(w)
    cq, cp, ck, cef = I.calibration_set(w)
    p, _, _ = I.query_params(w)
    assert cq.shape == q.shape and cq.dtype == q.dtype
    assert cq.min() >= 0 and cq.max() <= 255 and (cq == np.rint(cq)).all()
    assert not np.array_equal(cq, q) and not np.array_equal(cp, p)
    assert (cp > 0.5).all() and (cp <= 2.0).all()


def test_distance_error_against_fp64():
    """dist_err_vs_fp64 compares each returned distance with the FP64 L_p
    distance of its id: zero for exact values, the planted error otherwise,
    and absent ids (-1) are skipped."""
    import numpy as np

    import bench

    rng = np.random.default_rng(3)
    base = rng.integers(0, 256, size=(50, 8)).astype(np.float32)
    qs = rng.integers(0, 256, size=(3, 8)).astype(np.float32)
    p = np.array([0.5, 1.0, 1.7], np.float32)
    ids = np.array([[1, 2, -1], [3, 4, 5], [6, -1, -1]], np.int64)
    ref = np.zeros(ids.shape)
    for i in range(3):
        for j in range(3):
            if ids[i, j] >= 0:
                diff = np.abs(base[ids[i, j]].astype(np.float64) - qs[i].astype(np.float64))
                ref[i, j] = (diff ** float(p[i])).sum() ** (1.0 / float(p[i]))
    dist = ref.astype(np.float64)
    dist[1, 2] *= 1.0 + 3e-6
    worst, mean = bench.dist_err_vs_fp64(base, qs, p, ids, dist.astype(np.float32))
    f32 = np.abs(ref.astype(np.float32).astype(np.float64) - ref) / np.maximum(ref, 1e-30)
    assert worst[0] == max(f32[0, 0], f32[0, 1])
    assert abs(worst[1] - 3e-6) < 2e-7
    assert worst[2] == f32[2, 0]
    assert np.isfinite(mean).all()
