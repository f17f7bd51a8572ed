"""Fixed-p HNSW (Section 4.3's comparison): a graph built under the query's
own metric answers that p directly.  The L1.5 graph (metric 4) and graphs
under a general L_p (metric 5, p = 0.8 and 1.2): on 0/1 data every
|d_j|^p is exactly 0 or 1, so the GPU beam of a direct query equals the
oracle's search on the same graph id for id; on float data the answers carry
their exact L_p distances and reach the exact top-k; GPU-built graphs keep
HNSW's structure."""
import numpy as np
import pytest

import oracle
from paper_2605_02030_gb300 import inputs as I

from helpers import workload_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    import paper_2605_02030_gb300 as pkg
    pkg.build()
    from paper_2605_02030_gb300 import uhnsw
    uhnsw.load_library()
    return uhnsw


@pytest.mark.parametrize("qt", [32, 128])
def test_direct_p15_beam_equals_oracle(U, qt):
    r = np.random.default_rng(23)
    base = r.integers(0, 2, size=(2500, 32)).astype(np.float32)
    qs = r.integers(0, 2, size=(30, 32)).astype(np.float32)
    g15 = oracle.hnsw_build(base, 4, 8, 40, I.hnsw_levels(len(base), 8, 6))
    g2 = oracle.hnsw_build(base, 2, 8, 40, I.hnsw_levels(len(base), 8, 4))
    idx = U.Index(base, g15, g2, traverse_dtype="f16", metrics=(U.BASE_L15, U.BASE_L2))
    ef = 24
    p = np.full(len(qs), 1.5, np.float32)
    ids, dist, st = idx.search(torch.from_numpy(qs).cuda(), torch.from_numpy(p).cuda(), k=ef,
                               ef=ef, query_threads=qt, stats=True)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    for i in range(len(qs)):
        rid, rd, _ = oracle.hnsw_search(g15, base, qs[i], 4, ef, ef)
        np.testing.assert_array_equal(ids[i], rid, err_msg=f"query {i}")
        np.testing.assert_allclose(dist[i], rd ** (1 / 1.5), rtol=2e-6)
    assert (st[:, 6] == 1).all() and (st[:, 1] == 0).all()
    idx.close()


def test_gpu_built_l15_graph_structure(U):
    r = np.random.default_rng(24)
    base = r.normal(size=(3000, 48)).astype(np.float32)
    lv = I.hnsw_levels(len(base), 8, 6)
    g = U.build_graph(base, 4, 8, 40, lv, device="gpu")
    assert g["num_levels"] == lv.max() + 1 and lv[g["entry_point"]] == lv.max()
    for l, L in enumerate(g["levels"]):
        assert np.diff(L["offsets"]).max() <= (16 if l == 0 else 8)
        assert (lv[L["nbrs"]] >= l).all()


@pytest.fixture(scope="module")
def binary_lp():
    r = np.random.default_rng(29)
    base = r.integers(0, 2, size=(2500, 32)).astype(np.float32)
    qs = r.integers(0, 2, size=(30, 32)).astype(np.float32)
    g08 = oracle.hnsw_build(base, None, 8, 40, I.hnsw_levels(len(base), 8, 7), base_p=0.8)
    g2 = oracle.hnsw_build(base, 2, 8, 40, I.hnsw_levels(len(base), 8, 4))
    return base, qs, g08, g2


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("qt", [32, 128])
def test_direct_lp_beam_equals_oracle(U, binary_lp, dtype, qt):
    """p = 0.8 on a graph built under L0.8 (metric 5): answered directly, the
    beam id for id the oracle's, distances S^(1/0.8)."""
    base, qs, g08, g2 = binary_lp
    idx = U.Index(base, g08, g2, traverse_dtype=dtype, metrics=(U.BASE_LP, U.BASE_L2),
                  base_p=(0.8, 0.0))
    ef = 24
    p = np.full(len(qs), 0.8, np.float32)
    ids, dist, st = idx.search(torch.from_numpy(qs).cuda(), torch.from_numpy(p).cuda(), k=ef,
                               ef=ef, query_threads=qt, stats=True)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    for i in range(len(qs)):
        rid, rd, _ = oracle.hnsw_search(g08, base, qs[i], None, ef, ef, base_p=0.8)
        np.testing.assert_array_equal(ids[i], rid, err_msg=f"query {i}")
        np.testing.assert_allclose(dist[i], rd ** (1 / float(np.float32(0.8))), rtol=2e-6)
    assert (st[:, 6] == 1).all() and (st[:, 1] == 0).all()
    assert idx.device_status() == 0
    idx.close()


@pytest.mark.parametrize("qt", [32, 128])
def test_algorithm1_with_lp_graph_matches_oracle(U, binary_lp, qt):
    """Algorithm 1 over an (L0.8, L2) pair: p = 0.8 and p = 2 answered
    directly, every other p routed by the cutoff and verified; ids, distances
    and routes as the oracle's."""
    base, qs, g08, g2 = binary_lp
    idx = U.Index(base, g08, g2, traverse_dtype="f16", metrics=(U.BASE_LP, U.BASE_L2),
                  base_p=(0.8, 0.0))
    p = np.resize(np.array([0.3, 0.6, 0.8, 1.0, 1.3, 1.4, 1.41, 1.7, 2.0], np.float32), len(qs))
    ids, dist, st = idx.search(torch.from_numpy(qs).cuda(), torch.from_numpy(p).cuda(), k=10,
                               ef=40, query_threads=qt, stats=True)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    for i in range(len(qs)):
        rid, rd, rst = oracle.uhnsw_query(g08, g2, base, qs[i], float(p[i]), 10, 40,
                                          base_p=(0.8, 2.0))
        np.testing.assert_array_equal(ids[i], rid, err_msg=f"query {i} p={p[i]}")
        np.testing.assert_allclose(dist[i], rd, rtol=2e-5, err_msg=f"query {i} p={p[i]}")
    direct = (p == np.float32(0.8)) | (p == np.float32(2.0))
    assert (st[direct, 1] == 0).all() and (st[~direct, 1] > 0).all()
    slot = np.where(p <= np.float32(1.4), 1, 2)
    np.testing.assert_array_equal(st[:, 6], slot)
    assert idx.device_status() == 0
    idx.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_direct_lp_float_data(U, dtype):
    """p = 1.2 on float data, graph built by the library under L1.2 beside G2:
    every answer carries its exact L1.2 distance, ascending; recall@10 against
    the exact top-10 at least 0.9, and at least 8 of 10 ids shared with the
    oracle's direct search on the same graph."""
    w, base, qs, _, _, _ = workload_arrays("mixture10k", 4000, 60, 0.0)
    lv = I.graph_levels(w, 2)
    g12 = U.build_graph(base, U.BASE_LP, w.M, w.ef_construction, lv, threads=4, p=1.2)
    g2 = U.build_graph(base, U.BASE_L2, w.M, w.ef_construction, lv, threads=4)
    idx = U.Index(base, g12, g2, traverse_dtype=dtype, metrics=(U.BASE_LP, U.BASE_L2),
                  base_p=(1.2, 0.0))
    p = np.full(len(qs), 1.2, np.float32)
    ids, dist, st = idx.search(torch.from_numpy(qs).cuda(), torch.from_numpy(p).cuda(), k=10,
                               ef=64, persistent=True, use_graph=True, stats=True)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    gt, _ = oracle.exact_knn(base, qs, p, 10)
    pf = float(np.float32(1.2))
    hits = 0
    for i in range(len(qs)):
        ref = np.array([oracle.lp_sum(base[j], qs[i], pf) ** (1 / pf) for j in ids[i]])
        np.testing.assert_allclose(dist[i], ref, rtol=2e-5, err_msg=f"query {i}")
        assert np.all(np.diff(dist[i]) >= -2e-5 * dist[i, 1:])
        rid, _, _ = oracle.uhnsw_query(g12, g2, base, qs[i], pf, 10, 64, base_p=(1.2, 2.0))
        assert len(set(rid.tolist()) & set(ids[i].tolist())) >= 8, f"query {i} vs the oracle"
        hits += len(set(ids[i].tolist()) & set(gt[i].tolist()))
    assert hits / (10 * len(qs)) >= 0.9
    assert (st[:, 6] == 1).all()
    assert idx.device_status() == 0
    idx.close()


def test_gpu_built_lp_graph(U):
    """The GPU builder under L0.8: HNSW's structure, and direct p = 0.8
    search on it reaches recall@10 >= 0.9 at ef = 64."""
    w, base, qs, _, _, _ = workload_arrays("mixture10k", 4000, 60, 0.0)
    lv = I.graph_levels(w, 2)
    g = U.build_graph(base, U.BASE_LP, w.M, w.ef_construction, lv, device="gpu", p=0.8)
    assert g["num_levels"] == lv.max() + 1 and lv[g["entry_point"]] == lv.max()
    for l, L in enumerate(g["levels"]):
        assert np.diff(L["offsets"]).max() <= (2 * w.M if l == 0 else w.M)
        assert (lv[L["nbrs"]] >= l).all()
    g2 = U.build_graph(base, U.BASE_L2, w.M, w.ef_construction, lv, threads=4)
    idx = U.Index(base, g, g2, traverse_dtype="f16", metrics=(U.BASE_LP, U.BASE_L2),
                  base_p=(0.8, 0.0))
    p = np.full(len(qs), 0.8, np.float32)
    ids, _, _ = idx.search(torch.from_numpy(qs).cuda(), torch.from_numpy(p).cuda(), k=10, ef=64)
    gt, _ = oracle.exact_knn(base, qs, p, 10)
    ids = ids.cpu().numpy()
    hits = sum(len(set(ids[i].tolist()) & set(gt[i].tolist())) for i in range(len(qs)))
    assert hits / (10 * len(qs)) >= 0.9
    idx.close()
