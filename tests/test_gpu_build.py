"""HNSW construction on the GPU (uhnsw_build_graph_gpu): the graph keeps
every structural invariant of the published insertion, is the same on every
run, and searches as well as the host builder's graph (recall against the
oracle's exact answer at the same beam).  Graph construction is an input of
the query path, not part of it; like the multi-threaded host build it has no
exact reference ("parity unpinned"), so quality is what is compared."""
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


def check_structure(g, lv, M):
    n = len(lv)
    assert g["num_levels"] == lv.max() + 1
    assert lv[g["entry_point"]] == lv.max()
    for l, L in enumerate(g["levels"]):
        if l == 0:
            assert len(L["offsets"]) == n + 1
        else:
            np.testing.assert_array_equal(L["nodes"], np.nonzero(lv >= l)[0])
        deg = np.diff(L["offsets"])
        assert deg.max() <= (2 * M if l == 0 else M)
        nodes = np.arange(n) if l == 0 else L["nodes"]
        nb = L["nbrs"]
        assert ((nb >= 0) & (nb < n)).all() and (lv[nb] >= l).all()
        owner = np.repeat(nodes, deg)
        assert (owner != nb).all(), "self link"
        pairs = owner.astype(np.int64) * n + nb
        assert len(np.unique(pairs)) == len(pairs), "duplicate link"
    # layer 0 links the graph: almost every node is reachable from the entry
    L0 = g["levels"][0]
    seen = np.zeros(n, bool)
    seen[g["entry_point"]] = True
    fr = [g["entry_point"]]
    while fr:
        nxt = []
        for v in fr:
            for u in L0["nbrs"][L0["offsets"][v]:L0["offsets"][v + 1]]:
                if not seen[u]:
                    seen[u] = True
                    nxt.append(int(u))
        fr = nxt
    assert seen.mean() >= 0.98


def same_graph(a, b):
    if a["num_levels"] != b["num_levels"] or a["entry_point"] != b["entry_point"]:
        return False
    return all(np.array_equal(x[k], y[k]) for x, y in zip(a["levels"], b["levels"])
               for k in ("nodes", "offsets", "nbrs"))


@pytest.mark.parametrize("case", [("sift1m", 6000, 0.0, dict(M=12, ef_construction=64)),
                                  ("mixture10k", 4000, 0.0, dict(M=8, ef_construction=40))])
def test_gpu_build_structure_determinism_and_quality(U, case):
    name, n, grid, kw = case
    w, base, qs, p, _, _ = workload_arrays(name, n, 80, grid, **kw)
    graphs = {}
    for metric in (1, 2, 3):
        lv = I.graph_levels(w, metric)
        g = U.build_graph(base, metric, w.M, w.ef_construction, lv, device="gpu")
        check_structure(g, lv, w.M)
        again = U.build_graph(base, metric, w.M, w.ef_construction, lv, device="gpu")
        assert same_graph(g, again), f"metric {metric}: two GPU builds differ"
        host = U.build_graph(base, metric, w.M, w.ef_construction, lv, threads=4)
        graphs[metric] = (g, host)
    gt, _ = oracle.exact_knn(base, qs, p, 10)

    def recall(g1, g2, metrics, pq, truth):
        idx = U.Index(base, g1, g2, metrics=metrics)
        cut = 1.4 if metrics == U.U_HNSW else 0.6
        ids, _, _ = idx.search(torch.from_numpy(qs).cuda(), torch.from_numpy(pq).cuda(), k=10,
                               ef=32, cutoff=cut)
        ids = ids.cpu().numpy()
        idx.close()
        return np.mean([len(set(ids[i].tolist()) & set(truth[i].tolist())) / 10
                        for i in range(len(qs))])

    r_gpu = recall(graphs[1][0], graphs[2][0], U.U_HNSW, p, gt)
    r_host = recall(graphs[1][1], graphs[2][1], U.U_HNSW, p, gt)
    assert r_gpu >= r_host - 0.03, (r_gpu, r_host)
    # the L0.5 graph of U-HNSW-E, on queries with p in (0.2, 0.7]
    pe = (0.7 - 0.5 * np.random.default_rng(2).random(len(qs))).astype(np.float32)
    gte, _ = oracle.exact_knn(base, qs, pe, 10)
    r_gpu = recall(graphs[3][0], graphs[1][0], U.U_HNSW_E, pe, gte)
    r_host = recall(graphs[3][1], graphs[1][1], U.U_HNSW_E, pe, gte)
    assert r_gpu >= r_host - 0.03, (r_gpu, r_host)


def test_gpu_build_validation(U):
    base = np.zeros((10, 4), np.float32)
    lv = np.zeros(10, np.int32)
    with pytest.raises(U.UHNSWError):
        U.build_graph(base, 6, 4, 10, lv, device="gpu")
    with pytest.raises(ValueError):
        U.build_graph(base, U.BASE_LP, 4, 10, lv, device="gpu")     # L_p without its p
    with pytest.raises(U.UHNSWError):
        U.build_graph(base, U.BASE_LP, 4, 10, lv, device="gpu", p=2.5)
    with pytest.raises(U.UHNSWError):
        U.build_graph(base, 1, 4, 600, lv, device="gpu")       # efConstruction above 512
    lv[3] = -1
    with pytest.raises(U.UHNSWError):
        U.build_graph(base, 1, 4, 10, lv, device="gpu")
