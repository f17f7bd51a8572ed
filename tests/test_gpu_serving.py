"""Continuous-batching server (uhnsw_server_*): each request's result is the
same alone and inside the mix of concurrently running batches, admission keeps
the admitted search state within the budget, and latencies are recorded."""
import numpy as np
import pytest

from helpers import oracle_graphs, workload_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    import paper_2605_02030_gb300 as pkg
    pkg.build()
    from paper_2605_02030_gb300 import uhnsw as U
    w, base, qs, p, _, _ = workload_arrays("sift1m", 6000, 600, 0.0, M=12, ef_construction=80)
    g1, g2 = oracle_graphs("sift1m", 6000, 600, 0.0, M=12, ef_construction=80)
    idx = U.Index(base, g1, g2, traverse_dtype="f16")
    rng = np.random.default_rng(21)
    k = rng.choice([5, 10], size=len(qs)).astype(np.int32)
    ef = rng.choice([16, 24, 32, 48], size=len(qs)).astype(np.int32)
    yield U, idx, qs, p, k, ef
    idx.close()


def _alone(idx, q, p, k, ef, width=1):
    ids, dist, _ = idx.search(torch.from_numpy(q[None]).cuda(), torch.from_numpy(p[None]).cuda(),
                              k=int(k), ef=int(ef), k_max=10, width=width)
    return ids.cpu().numpy()[0], dist.cpu().numpy()[0]


@pytest.mark.parametrize("width", [1, 3])
def test_results_equal_alone_and_in_the_mix(served, width):
    U, idx, qs, p, k, ef = served
    arrivals = np.cumsum(np.random.default_rng(3).exponential(10.0, size=len(qs)))  # ~100k QPS
    srv = U.Server(idx, max_batch=32, streams=4, k_max=10, ef_max=64, max_delay_us=50,
                   width=width)
    ids, dist, lat = srv.replay(qs, p, k, ef, arrivals)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(qs) and st["error"] == 0
    assert st["batches"] > 1 and st["peak_inflight"] > 1
    assert (lat > 0).all() and st["p99_us"] >= st["p50_us"] > 0
    for i in range(len(qs)):
        a_ids, a_d = _alone(idx, qs[i], p[i], k[i], ef[i], width)
        np.testing.assert_array_equal(ids[i], a_ids, err_msg=f"request {i}")
        np.testing.assert_array_equal(dist[i], a_d, err_msg=f"request {i}")
    assert idx.device_status() == 0


def test_admission_respects_state_budget(served):
    U, idx, qs, p, k, ef = served
    n = 200
    arrivals = np.zeros(n)                       # everything arrives at once
    # one query per batch and one stream: the peak state is one query's state
    srv = U.Server(idx, max_batch=1, streams=1, k_max=10, ef_max=64)
    srv.replay(qs[:n], p[:n], 10, 64, arrivals)
    one = srv.stats()["peak_state"]
    srv.close()
    assert one > 0
    budget = 5 * one
    srv = U.Server(idx, max_batch=64, streams=4, k_max=10, ef_max=64, state_budget=budget)
    ids, dist, lat = srv.replay(qs[:n], p[:n], 10, 64, arrivals)
    st = srv.stats()
    srv.close()
    assert st["completed"] == n and st["peak_state"] <= budget
    assert st["peak_inflight"] <= 5 and st["batches"] >= n // 5
    for i in range(0, n, 17):
        a_ids, a_d = _alone(idx, qs[i], p[i], 10, 64)
        np.testing.assert_array_equal(ids[i], a_ids)
        np.testing.assert_array_equal(dist[i], a_d)


def test_submit_poll_wait_and_limits(served):
    U, idx, qs, p, k, ef = served
    srv = U.Server(idx, max_batch=8, streams=2, k_max=10, ef_max=64)
    with pytest.raises(U.UHNSWError):
        srv.submit(qs[0], 0.0, 10, 32)           # p outside (0, 2]
    with pytest.raises(U.UHNSWError):
        srv.submit(qs[0], 1.2, 11, 32)           # k above the server's k_max
    t = srv.submit(qs[3], p[3], 10, 32)
    ids, dist = srv.wait(t, 10)
    a_ids, a_d = _alone(idx, qs[3], p[3], 10, 32)
    np.testing.assert_array_equal(ids, a_ids)
    srv.close()
