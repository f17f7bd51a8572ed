"""Persistent searches on several streams.  Each stream has a queue of its own,
so batches issued back to back on two streams overlap on the GPU; every
batch's result must equal the same batch searched alone on one stream, with
fixed and per-query beams (one launch per beam bucket), with CUDA-graph
replay, and after a stream's queue workspace has grown under a captured
graph."""
import numpy as np
import pytest

from helpers import oracle_graphs, workload_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2605_02030_gb300 as pkg
    pkg.build()
    from paper_2605_02030_gb300 import uhnsw as U
    w, base, qs, p, _, _ = workload_arrays("sift1m", 6000, 600, 0.0, M=12, ef_construction=80)
    g1, g2 = oracle_graphs("sift1m", 6000, 600, 0.0, M=12, ef_construction=80)
    idx = U.Index(base, g1, g2, traverse_dtype="f16")
    q = torch.from_numpy(qs).cuda()
    pd = torch.from_numpy(p).cuda()
    ef_q = torch.from_numpy(np.random.default_rng(5).choice([24, 48, 96, 160], size=len(qs))
                            .astype(np.int32)).cuda()
    yield U, idx, q, pd, ef_q
    idx.close()


def _alone(idx, q, pd, ef, **kw):
    ids, dist, _ = idx.search(q, pd, k=10, ef=ef, persistent=True, **kw)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("per_query_ef", [False, True])
@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("width", [1, 2])
def test_overlapping_persistent_batches_equal_alone(setup, per_query_ef, use_graph, width):
    U, idx, q, pd, ef_q = setup
    ef = ef_q if per_query_ef else 40
    kw = dict(width=width, ef_max=160 if per_query_ef else 0)
    parts = [slice(0, 600), slice(100, 400), slice(250, 600)]
    ref = []
    for sl in parts:
        e = ef[sl] if per_query_ef else ef
        ref.append(_alone(idx, q[sl], pd[sl], e, **kw))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = {}
    torch.cuda.synchronize()
    for rep in range(3):             # later repetitions replay captured graphs
        for j, sl in enumerate(parts):
            st = streams[j % 2]
            n = sl.stop - sl.start
            out = (torch.empty((n, 10), dtype=torch.int64, device="cuda"),
                   torch.empty((n, 10), dtype=torch.float32, device="cuda"))
            e = ef[sl] if per_query_ef else ef
            with torch.cuda.stream(st):
                idx.search(q[sl], pd[sl], k=10, ef=e, persistent=True, use_graph=use_graph,
                           stream=st, out=out, **kw)
            outs[(rep, j)] = out
    torch.cuda.synchronize()
    for (rep, j), (ids, dist) in outs.items():
        np.testing.assert_array_equal(ids.cpu().numpy(), ref[j][0], err_msg=f"rep {rep} part {j}")
        np.testing.assert_array_equal(dist.cpu().numpy(), ref[j][1], err_msg=f"rep {rep} part {j}")
    assert idx.device_status() == 0


def test_graph_replay_after_queue_growth(setup):
    U, idx, q, pd, _ = setup
    st = torch.cuda.Stream()
    small_ref = _alone(idx, q[:50], pd[:50], 32)
    big_ref = _alone(idx, q, pd, 32)
    out_s = (torch.empty((50, 10), dtype=torch.int64, device="cuda"),
             torch.empty((50, 10), dtype=torch.float32, device="cuda"))
    out_b = (torch.empty((600, 10), dtype=torch.int64, device="cuda"),
             torch.empty((600, 10), dtype=torch.float32, device="cuda"))
    with torch.cuda.stream(st):
        # a graph captured on a fresh stream's small workspace, then a batch
        # that grows that workspace, then the small graph replayed
        idx.search(q[:50], pd[:50], k=10, ef=32, persistent=True, use_graph=True, stream=st,
                   out=out_s)
        idx.search(q, pd, k=10, ef=32, persistent=True, use_graph=True, stream=st, out=out_b)
        for _ in range(2):
            out_s[0].fill_(-7)
            idx.search(q[:50], pd[:50], k=10, ef=32, persistent=True, use_graph=True, stream=st,
                       out=out_s)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out_s[0].cpu().numpy(), small_ref[0])
    np.testing.assert_array_equal(out_s[1].cpu().numpy(), small_ref[1])
    np.testing.assert_array_equal(out_b[0].cpu().numpy(), big_ref[0])
    assert idx.device_status() == 0


def test_server_with_persistent_launches(setup):
    U, idx, q, pd, _ = setup
    qs = q.cpu().numpy()
    p = pd.cpu().numpy()
    arrivals = np.cumsum(np.random.default_rng(4).exponential(5.0, size=len(qs)))
    srv = U.Server(idx, max_batch=64, streams=4, k_max=10, ef_max=64, max_delay_us=50,
                   persistent=True)
    ids, dist, lat = srv.replay(qs, p, 10, 48, arrivals)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(qs) and st["error"] == 0 and st["batches"] > 1
    ref_ids, ref_d = _alone(idx, q, pd, 48)
    np.testing.assert_array_equal(ids, ref_ids)
    np.testing.assert_array_equal(dist, ref_d)
    assert idx.device_status() == 0


def test_host_async_on_two_streams_equals_sync(setup):
    U, idx, q, pd, _ = setup
    qs = q.cpu().numpy()
    p = pd.cpu().numpy()
    ref_ids, ref_d = idx.search_host(qs, p, k=10, ef=40, persistent=True, width=2)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    parts = [slice(0, 600), slice(50, 350), slice(300, 600), slice(0, 200)]
    ins = [(pin(qs[sl]), pin(p[sl])) for sl in parts]
    outs = [(pin(np.zeros((sl.stop - sl.start, 10), np.int64)),
             pin(np.zeros((sl.stop - sl.start, 10), np.float32))) for sl in parts]
    torch.cuda.synchronize()
    for rep in range(2):
        for j, sl in enumerate(parts):
            outs[j][0].fill(-5)
            idx.search_host(ins[j][0], ins[j][1], k=10, ef=40, persistent=True, width=2,
                            out=outs[j], stream=streams[j % 2], wait=False)
        torch.cuda.synchronize()
        for j, sl in enumerate(parts):
            np.testing.assert_array_equal(outs[j][0], ref_ids[sl], err_msg=f"rep {rep} part {j}")
            np.testing.assert_array_equal(outs[j][1], ref_d[sl], err_msg=f"rep {rep} part {j}")
    # no temporaries may back an asynchronous call
    with pytest.raises(ValueError):
        idx.search_host(qs.astype(np.float64), p, k=10, ef=40, out=outs[0], wait=False)
    with pytest.raises(ValueError):
        idx.search_host(qs[:, ::2], p, k=10, ef=40, out=outs[0], wait=False)
    with pytest.raises(ValueError):
        idx.search_host(ins[0][0], ins[0][1], k=10, ef=40, wait=False)
    assert idx.device_status() == 0


@pytest.mark.parametrize("width", [1, 2])
def test_batch_size_shape_changes_no_result(setup, width):
    """A batch with at least as many queries as the GPU has warp slots runs
    2 rows per team and round, a smaller one 3 rows; every row's sum takes
    the same order either way, so the results are identical."""
    U, idx, q, pd, _ = setup
    slots = torch.cuda.get_device_properties(0).multi_processor_count * 24
    reps = slots // q.shape[0] + 1
    big_q = q.repeat(reps, 1)
    big_p = pd.repeat(reps)
    assert big_q.shape[0] >= slots
    ids_b, d_b, _ = idx.search(big_q, big_p, k=10, ef=48, width=width, persistent=True)
    ids_s, d_s, _ = idx.search(q, pd, k=10, ef=48, width=width, persistent=True)
    torch.cuda.synchronize()
    ids_b = ids_b.cpu().numpy().reshape(reps, q.shape[0], 10)
    d_b = d_b.cpu().numpy().reshape(reps, q.shape[0], 10)
    for r in range(reps):
        np.testing.assert_array_equal(ids_b[r], ids_s.cpu().numpy())
        np.testing.assert_array_equal(d_b[r], d_s.cpu().numpy())
    assert idx.device_status() == 0


@pytest.mark.parametrize("use_graph", [False, True])
def test_threads_sharing_one_stream(setup, use_graph):
    """Persistent searches issued from several host threads on one stream
    keep each call's queue reset, ordering and launch together: every
    result equals the slice searched alone."""
    from concurrent.futures import ThreadPoolExecutor

    U, idx, q, pd, _ = setup
    ref_ids, ref_d = _alone(idx, q, pd, 40, width=2)
    st = torch.cuda.Stream()
    parts = [slice(a, a + 150) for a in (0, 150, 300, 450)]
    outs = {}

    def work(j):
        sl = parts[j]
        for r in range(5):
            out = (torch.empty((150, 10), dtype=torch.int64, device="cuda"),
                   torch.empty((150, 10), dtype=torch.float32, device="cuda"))
            idx.search(q[sl], pd[sl], k=10, ef=40, width=2, persistent=True,
                       use_graph=use_graph, stream=st, out=out)
            outs[(j, r)] = out

    torch.cuda.synchronize()
    with ThreadPoolExecutor(max_workers=4) as ex:
        list(ex.map(work, range(4)))
    torch.cuda.synchronize()
    for (j, r), (ids, dist) in outs.items():
        np.testing.assert_array_equal(ids.cpu().numpy(), ref_ids[parts[j]], err_msg=f"{j} {r}")
        np.testing.assert_array_equal(dist.cpu().numpy(), ref_d[parts[j]], err_msg=f"{j} {r}")
    assert idx.device_status() == 0
