"""U-HNSW-E (Section 4.5) on the GPU: graphs under L0.5 (G0.5) and L1 (G1),
cutoff 0.6, p in [0.2, 1].  Parity with the oracle's Algorithm 1 run with the
same graphs and base metrics.

0/1 data makes every |d_j|^p exactly 0 or 1, so every FP32 sum on the GPU is
exact (L0.5 traversal included) and the beam of a direct p = 0.5 query equals
the oracle's HNSW search on G0.5 id for id.  Float data (a 1/16 grid) checks
the properties that hold at any size: each returned id carries its own FP64
L_p distance, lists ascend, and recall against the exact answer stays high."""
import numpy as np
import pytest

import oracle
from paper_2605_02030_gb300 import inputs as I

from helpers import workload_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
E = dict(cutoff=0.6)


@pytest.fixture(scope="module")
def U():
    import paper_2605_02030_gb300 as pkg
    pkg.build()
    from paper_2605_02030_gb300 import uhnsw
    uhnsw.load_library()
    return uhnsw


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def binary_case():
    r = np.random.default_rng(17)
    base = r.integers(0, 2, size=(3000, 32)).astype(np.float32)
    qs = r.integers(0, 2, size=(40, 32)).astype(np.float32)
    g05 = oracle.hnsw_build(base, 3, 8, 40, I.hnsw_levels(len(base), 8, 5))
    g1 = oracle.hnsw_build(base, 1, 8, 40, I.hnsw_levels(len(base), 8, 3))
    return base, qs, g05, g1


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("qt", [32, 128])
def test_direct_p05_beam_equals_oracle(U, binary_case, dtype, qt):
    base, qs, g05, g1 = binary_case
    idx = U.Index(base, g05, g1, traverse_dtype=dtype, metrics=U.U_HNSW_E)
    nq, ef = len(qs), 32
    p = np.full(nq, 0.5, np.float32)
    ids, dist, st = idx.search(dev(qs), dev(p), k=ef, ef=ef, query_threads=qt, stats=True, **E)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    for i in range(nq):
        rid, rd, _ = oracle.hnsw_search(g05, base, qs[i], 3, ef, ef)
        np.testing.assert_array_equal(ids[i], rid, err_msg=f"query {i}")
        np.testing.assert_allclose(dist[i], rd ** 2, rtol=0, atol=0)   # S^(1/0.5)
    assert (st[:, 6] == 1).all() and (st[:, 1] == 0).all()
    assert idx.device_status() == 0
    idx.close()


@pytest.mark.parametrize("qt", [32, 128])
def test_algorithm1_e_matches_oracle_on_exact_data(U, binary_case, qt):
    base, qs, g05, g1 = binary_case
    idx = U.Index(base, g05, g1, traverse_dtype="f16", metrics=U.U_HNSW_E)
    nq = len(qs)
    p = np.resize(np.array([0.2, 0.35, 0.5, 0.6, 0.61, 0.75, 0.9, 1.0], np.float32), nq)
    ids, dist, st = idx.search(dev(qs), dev(p), k=10, ef=40, query_threads=qt, stats=True, **E)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    for i in range(nq):
        rid, rd, rst = oracle.uhnsw_query(g05, g1, base, qs[i], float(p[i]), 10, 40, cutoff=0.6,
                                          metrics=(3, 1))
        np.testing.assert_array_equal(ids[i], rid, err_msg=f"query {i} p={p[i]}")
        np.testing.assert_allclose(dist[i], rd, rtol=2e-5, err_msg=f"query {i} p={p[i]}")
    slot = np.where(p <= np.float32(0.6), 1, 2)
    slot[p == np.float32(1.0)] = 2
    np.testing.assert_array_equal(st[:, 6], slot)
    assert idx.device_status() == 0
    idx.close()


def test_algorithm1_e_float_data(U):
    w, base, qs, _, _, _ = workload_arrays("mixture10k", 4000, 60, 1 / 16)
    g05 = oracle.hnsw_build(base, 3, w.M, w.ef_construction, I.graph_levels(w, 3))
    g1 = oracle.hnsw_build(base, 1, w.M, w.ef_construction, I.graph_levels(w, 1))
    idx = U.Index(base, g05, g1, traverse_dtype="f32", metrics=U.U_HNSW_E)
    p = (0.7 - 0.5 * np.random.default_rng(3).random(len(qs))).astype(np.float32)
    p[:2] = [0.5, 1.0]
    ids, dist, _ = idx.search(dev(qs), dev(p), k=10, ef=64, persistent=True, use_graph=True, **E)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    gt, _ = oracle.exact_knn(base, qs, p, 10)
    hits = 0
    for i in range(len(qs)):
        rid, _, _ = oracle.uhnsw_query(g05, g1, base, qs[i], float(p[i]), 10, 64, cutoff=0.6,
                                       metrics=(3, 1))
        hits += len(set(ids[i].tolist()) & set(gt[i].tolist()))
        ref = np.array([oracle.lp_sum(base[j], qs[i], float(p[i])) ** (1 / float(p[i]))
                        for j in ids[i]])
        np.testing.assert_allclose(dist[i], ref, rtol=2e-5, err_msg=f"query {i}")
        assert np.all(np.diff(dist[i]) >= -2e-5 * dist[i, 1:])
        assert len(set(rid.tolist()) & set(ids[i].tolist())) >= 8, f"query {i} vs the oracle"
    assert hits / (10 * len(qs)) >= 0.9
    assert idx.device_status() == 0
    idx.close()


def test_load_rejects_bad_base_metrics(U, binary_case):
    base, qs, g05, g1 = binary_case
    for metrics in ((1, 3), (2, 2), (4, 1)):
        with pytest.raises(U.UHNSWError):
            U.Index(base, g05, g1, metrics=metrics)
