"""The small plain U-HNSW configuration at its full size: 10,000 x 32
Gaussian-mixture base vectors (16 centres ~ N(0, 4I), unit noise), 100
queries with p ~ U(0.5, 2], k = 10, graphs M = 16 and efConstruction = 100,
ef = 64, FP32 rows.  The values are rounded to a 1/16 grid, so that every
FP32 base distance is an exact sum: the beam then equals the oracle's
search id for id, and Algorithm 1 matches the oracle's within the
verification bar."""
import numpy as np
import pytest

import oracle

from helpers import check_topk, oracle_graphs, workload_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    import paper_2605_02030_gb300 as pkg
    pkg.build()
    from paper_2605_02030_gb300 import uhnsw as U
    w, base, qs, p, k, ef = workload_arrays("mixture10k", 10_000, 100, 1 / 16)
    g1, g2 = oracle_graphs("mixture10k", 10_000, 100, 1 / 16)
    idx = U.Index(base, g1, g2, traverse_dtype="f32")
    yield U, w, base, qs, p, g1, g2, idx
    idx.close()


@pytest.mark.parametrize("qt", [32, 128])
def test_full_beam_equals_oracle(case, qt):
    U, w, base, qs, p, g1, g2, idx = case
    nq, ef = len(qs), w.ef
    for pp, metric, g in ((1.0, 1, g1), (2.0, 2, g2)):
        pv = np.full(nq, pp, np.float32)
        ids, _, _ = idx.search(torch.from_numpy(qs).cuda(), torch.from_numpy(pv).cuda(), k=ef,
                               ef=ef, query_threads=qt)
        ids = ids.cpu().numpy()
        for i in range(nq):
            rid, _, _ = oracle.hnsw_search(g, base, qs[i], metric, ef, ef)
            np.testing.assert_array_equal(ids[i], rid, err_msg=f"p={pp} query {i}")


@pytest.mark.parametrize("persistent", [False, True])
def test_algorithm1_matches_oracle_and_recall(case, persistent):
    U, w, base, qs, p, g1, g2, idx = case
    ids, dist, st = idx.search(torch.from_numpy(qs).cuda(), torch.from_numpy(p).cuda(), k=w.k,
                               ef=w.ef, persistent=persistent, stats=True)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    assert (st[:, 5] == 0).all()
    for i in range(len(qs)):
        rid, _, _ = oracle.uhnsw_query(g1, g2, base, qs[i], float(p[i]), w.k, w.ef)
        check_topk(base, qs[i], p[i], ids[i], dist[i], rid, w.k, f"query {i} p={p[i]}")
    gt, _ = oracle.exact_knn(base, qs, p, w.k)
    rec = np.mean([len(set(ids[i].tolist()) & set(gt[i].tolist())) / w.k for i in range(len(qs))])
    assert rec >= 0.9
