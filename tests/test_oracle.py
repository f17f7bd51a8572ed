"""Pins for the CPU oracle (no GPU): closed forms, library routines, hand-
derived HNSW graphs and invariants that a plausible mistake in the oracle
(a dropped term, a wrong exponent or sign, a flipped comparison, a
transposed operand, a wrong tie rule) would break."""
import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.spatial.distance import cdist

import oracle
from paper_2605_02030_gb300 import inputs as I


def rng(s=0):
    return np.random.default_rng(s)


# ----------------------------------------------------------------- distances
def test_lp_sum_hand_values():
    x = np.array([0.0, 0.0], np.float32)
    q = np.array([1.0, 4.0], np.float32)
    assert oracle.lp_sum(x, q, 0.5) == 3.0          # 1 + 2
    assert oracle.lp_sum(x, q, 1.0) == 5.0
    assert oracle.lp_sum(x, q, 1.5) == 9.0          # 1 + 8
    assert oracle.lp_sum(x, q, 2.0) == 17.0
    assert oracle.lp_sum(q, x, 0.5) == 3.0          # symmetric
    assert oracle.lp_sum(x, x, 0.7) == 0.0          # |0|^p = 0
    assert oracle.base_dist(x, q, 1) == 5.0
    assert oracle.base_dist(x, q, 2) == 17.0


@pytest.mark.parametrize("p", [0.5, 0.63, 1.0, 1.37, 1.5, 2.0])
def test_lp_sum_matches_scipy_minkowski(p):
    r = rng(1)
    x = r.normal(size=(20, 37)).astype(np.float32)
    q = r.normal(size=(37,)).astype(np.float32)
    ref = cdist(x.astype(np.float64), q[None].astype(np.float64), "minkowski", p=p)[:, 0] ** p
    got = np.array([oracle.lp_sum(xi, q, p) for xi in x])
    np.testing.assert_allclose(got, ref, rtol=1e-12)
    l1 = cdist(x.astype(np.float64), q[None].astype(np.float64), "cityblock")[:, 0]
    l2 = cdist(x.astype(np.float64), q[None].astype(np.float64), "sqeuclidean")[:, 0]
    np.testing.assert_allclose([oracle.base_dist(xi, q, 1) for xi in x], l1, rtol=1e-12)
    np.testing.assert_allclose([oracle.base_dist(xi, q, 2) for xi in x], l2, rtol=1e-12)


def test_lp_norm_inequalities():
    """Norm equivalence in finite dimension (Section 3.1): for p < r,
    ||v||_r <= ||v||_p <= d^(1/p - 1/r) ||v||_r."""
    r = rng(2)
    d = 48
    ps = [0.5, 0.7, 1.0, 1.3, 1.5, 2.0]
    for _ in range(20):
        x = r.normal(size=d).astype(np.float32)
        q = r.normal(size=d).astype(np.float32)
        norms = [oracle.lp_sum(x, q, p) ** (1 / p) for p in ps]
        for i in range(len(ps) - 1):
            p, rr = ps[i], ps[i + 1]
            assert norms[i] >= norms[i + 1] * (1 - 1e-12)
            assert norms[i] <= d ** (1 / p - 1 / rr) * norms[i + 1] * (1 + 1e-12)


def test_lp_sum_homogeneity_and_translation():
    r = rng(3)
    x = r.integers(-8, 8, size=16).astype(np.float32)
    q = r.integers(-8, 8, size=16).astype(np.float32)
    for p in (0.5, 0.9, 1.7):
        s = oracle.lp_sum(x, q, p)
        assert oracle.lp_sum(4 * x, 4 * q, p) == pytest.approx(4 ** p * s, rel=1e-12)
        assert oracle.lp_sum(x + 3, q + 3, p) == pytest.approx(s, rel=1e-12)


# ----------------------------------------------------------------- O1
@pytest.mark.parametrize("p", [1.0, 1.25, 1.5, 2.0])
def test_exact_knn_matches_kdtree(p):
    """An independent exact k-NN algorithm (k-d tree, Minkowski p >= 1)."""
    r = rng(4)
    base = r.normal(size=(600, 6)).astype(np.float32)
    qs = r.normal(size=(15, 6)).astype(np.float32)
    ids, S = oracle.exact_knn(base, qs, p, 7)
    dist, kid = cKDTree(base.astype(np.float64)).query(qs.astype(np.float64), k=7, p=p)
    np.testing.assert_array_equal(ids, kid)
    np.testing.assert_allclose(S ** (1 / p), dist, rtol=1e-10)


@pytest.mark.parametrize("p", [0.5, 0.55, 0.8])
def test_exact_knn_fractional_p_bruteforce(p):
    r = rng(5)
    base = r.normal(size=(300, 9)).astype(np.float32)
    qs = r.normal(size=(10, 9)).astype(np.float32)
    ids, S = oracle.exact_knn(base, qs, p, 5)
    pf = float(np.float32(p))            # the oracle takes p as the FP32 query value
    D = cdist(qs.astype(np.float64), base.astype(np.float64), "minkowski", p=pf) ** pf
    for i in range(len(qs)):
        order = np.lexsort((np.arange(len(base)), D[i]))[:5]
        np.testing.assert_array_equal(ids[i], order)
        np.testing.assert_allclose(S[i], D[i, order], rtol=1e-12)


def test_exact_knn_ties_and_padding():
    base = np.array([[0.0], [1.0], [1.0], [0.0]], np.float32)
    ids, S = oracle.exact_knn(base, np.zeros((1, 1), np.float32), 1.0, 3)
    assert ids.tolist() == [[0, 3, 1]]                  # equal S -> ids ascending
    assert S.tolist() == [[0.0, 0.0, 1.0]]
    ids, S = oracle.exact_knn(base[:2], np.zeros((1, 1), np.float32), 0.5, 4)
    assert ids.tolist() == [[0, 1, -1, -1]]
    assert np.isinf(S[0, 2:]).all()


# ----------------------------------------------------------------- O2 (heuristic + build)
def test_heuristic_line():
    base = np.array([[0.0], [1.0], [2.0], [3.0]], np.float32)
    # base point is node 0; candidates 1, 2, 3 at L1 distances 1, 2, 3
    sel = oracle.select_heuristic(base, [1, 2, 3], [1.0, 2.0, 3.0], 3, metric=1)
    assert sel.tolist() == [1]


def test_heuristic_plane_and_limit():
    base = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [2, 0]], np.float32)
    cand, cd = [1, 2, 3, 4], [1.0, 1.0, 1.0, 4.0]       # squared L2 to node 0
    assert oracle.select_heuristic(base, cand, cd, 4, metric=2).tolist() == [1, 2, 3]
    assert oracle.select_heuristic(base, cand, cd, 2, metric=2).tolist() == [1, 2]


def test_heuristic_tie_rule():
    """e equidistant from the base point and a kept neighbour is dropped:
    a candidate is kept only if strictly nearer to the base point."""
    base = np.array([[0.0], [2.0], [1.0]], np.float32)   # b=0, r=node1 at 2, e=node2 at 1
    # candidates sorted by distance to b: node2 (1) first -> kept; then node1 (2):
    # dist(node1, node2) = 1 < 2 -> dropped
    assert oracle.select_heuristic(base, [2, 1], [1.0, 2.0], 2, 1).tolist() == [2]
    # r kept first (closer), then e with dist(e, b) == dist(e, r)
    base = np.array([[0.0], [1.0], [2.0]], np.float32)   # b=0; r=1 (d 1); e=2 (d 2), dist(e,r)=1
    assert oracle.select_heuristic(base, [1, 2], [1.0, 2.0], 2, 1).tolist() == [1]
    base2 = np.array([[0.0, 0.0], [-1.0, 0.0], [1.0, 0.0]], np.float32)
    # e=(1,0): d(e,b)=1, r=(-1,0): d(e,r)=2 -> kept
    assert oracle.select_heuristic(base2, [1, 2], [1.0, 1.0], 2, 1).tolist() == [1, 2]
    base3 = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 0.5]], np.float32)
    # L1: r=(1,0) d 1, e=(0.5,0.5) d 1 -> d(e,r) = 1 == d(e,b) -> dropped (strict rule)
    assert oracle.select_heuristic(base3, [1, 2], [1.0, 1.0], 2, 1).tolist() == [1]


def _lists(g, l):
    lv = g["levels"][l]
    return {int(v): lv["nbrs"][lv["offsets"][i]:lv["offsets"][i + 1]].tolist()
            for i, v in enumerate(lv["nodes"])}


def test_build_chain_by_hand():
    """Points 0..5 on a line, one layer, M=2: each insertion links to its
    left neighbour only (the heuristic drops the others), giving a chain."""
    base = np.arange(6, dtype=np.float32)[:, None]
    g = oracle.hnsw_build(base, 1, M=2, ef_construction=10, levels=np.zeros(6, np.int32), M0=4)
    assert g["num_levels"] == 1 and g["entry_point"] == 0
    assert _lists(g, 0) == {0: [1], 1: [0, 2], 2: [1, 3], 3: [2, 4], 4: [3, 5], 5: [4]}


def test_build_shrink_by_hand():
    """Node 0 at the origin gets a third link with M0=2 and is pruned by the
    heuristic over three equidistant neighbours (ties broken by id)."""
    base = np.array([[0, 0], [4, 0], [-4, 0], [0, 4]], np.float32)
    g = oracle.hnsw_build(base, 2, M=2, ef_construction=10, levels=np.zeros(4, np.int32), M0=2)
    assert _lists(g, 0) == {0: [1, 2], 1: [0], 2: [0], 3: [0]}


def test_build_levels_by_hand():
    base = np.arange(4, dtype=np.float32)[:, None]
    g = oracle.hnsw_build(base, 1, M=2, ef_construction=10, levels=np.array([0, 1, 0, 0], np.int32),
                          M0=4)
    assert g["num_levels"] == 2 and g["entry_point"] == 1
    assert _lists(g, 0) == {0: [1], 1: [0, 2], 2: [1, 3], 3: [2]}
    assert _lists(g, 1) == {1: []}


def _bfs_reach(g, start):
    lists = g["levels"][0]
    seen = np.zeros(g["n"], bool)
    seen[start] = True
    frontier = [start]
    while frontier:
        nxt = []
        for v in frontier:
            for u in lists["nbrs"][lists["offsets"][v]:lists["offsets"][v + 1]]:
                if not seen[u]:
                    seen[u] = True
                    nxt.append(int(u))
        frontier = nxt
    return seen


@pytest.fixture(scope="module")
def mixture_small():
    w = I.WORKLOADS["mixture10k"].scaled(n=3000, nq=30)
    base = I.base_vectors(w)
    qs = I.query_vectors(w)
    p, k, ef = I.query_params(w)
    g1 = oracle.hnsw_build(base, 1, w.M, w.ef_construction, I.graph_levels(w, 1))
    g2 = oracle.hnsw_build(base, 2, w.M, w.ef_construction, I.graph_levels(w, 2))
    return w, base, qs, p, g1, g2


def test_build_structure(mixture_small):
    w, base, qs, p, g1, g2 = mixture_small
    for metric, g in ((1, g1), (2, g2)):
        levels = I.graph_levels(w, metric)
        assert g["num_levels"] == levels.max() + 1
        assert levels[g["entry_point"]] == levels.max()
        for l, lv in enumerate(g["levels"]):
            np.testing.assert_array_equal(lv["nodes"], np.nonzero(levels >= l)[0])
            deg = np.diff(lv["offsets"])
            assert deg.max() <= (g["max_degree0"] if l == 0 else g["max_degree"])
            for i, v in enumerate(lv["nodes"]):
                nb = lv["nbrs"][lv["offsets"][i]:lv["offsets"][i + 1]]
                assert v not in nb and len(set(nb.tolist())) == len(nb)
                assert (levels[nb] >= l).all()
        assert _bfs_reach(g, g["entry_point"]).all()


# ----------------------------------------------------------------- O3
def test_search_full_beam_is_exact(mixture_small):
    """With ef >= N on a connected layer 0 the beam visits every node, so the
    first t results are the exact base-metric top-t."""
    w, base, qs, p, g1, g2 = mixture_small
    for metric, g, name in ((1, g1, "cityblock"), (2, g2, "sqeuclidean")):
        D = cdist(qs[:5].astype(np.float64), base.astype(np.float64), name)
        for i in range(5):
            ids, dd, nd = oracle.hnsw_search(g, base, qs[i], metric, ef=len(base), t=20)
            order = np.lexsort((np.arange(len(base)), D[i]))[:20]
            np.testing.assert_array_equal(ids, order)
            np.testing.assert_allclose(dd, D[i, order], rtol=1e-12)
            assert nd >= len(base)


def test_search_greedy_chain_by_hand():
    base = np.arange(6, dtype=np.float32)[:, None]
    g = oracle.hnsw_build(base, 1, M=2, ef_construction=10, levels=np.zeros(6, np.int32), M0=4)
    # ef=1 from entry 0 toward 4.2 walks the chain and stops at 4
    ids, dd, nd = oracle.hnsw_search(g, base, np.array([4.2], np.float32), 1, ef=1, t=1)
    assert ids.tolist() == [4]
    assert dd[0] == pytest.approx(0.2, rel=1e-6)
    ids, dd, nd = oracle.hnsw_search(g, base, np.array([4.2], np.float32), 1, ef=3, t=3)
    assert ids.tolist() == [4, 5, 3]


def test_search_results_sorted_and_recall(mixture_small):
    w, base, qs, p, g1, g2 = mixture_small
    D = cdist(qs.astype(np.float64), base.astype(np.float64), "cityblock")
    hits = 0
    for i in range(len(qs)):
        ids, dd, _ = oracle.hnsw_search(g1, base, qs[i], 1, ef=32, t=10)
        assert (np.diff(dd) >= 0).all()
        hits += len(set(ids.tolist()) & set(np.argsort(D[i])[:10].tolist()))
    assert hits / (10 * len(qs)) >= 0.95


# ----------------------------------------------------------------- O4
def test_verify_exact_bruteforce_and_abandon():
    r = rng(6)
    base = r.normal(size=(500, 24)).astype(np.float32)
    q = r.normal(size=24).astype(np.float32)
    cand = r.choice(500, size=80, replace=False).astype(np.int32)
    for p in (0.5, 0.77, 1.5, 1.93):
        pf = float(np.float32(p))
        S = cdist(q[None].astype(np.float64), base[cand].astype(np.float64), "minkowski", p=pf)[0] ** pf
        order = np.lexsort((cand, S))[:10]
        a_ids, a_S, a_terms = oracle.verify_exact(base, q, p, cand, 10, abandon=True)
        b_ids, b_S, b_terms = oracle.verify_exact(base, q, p, cand, 10, abandon=False)
        np.testing.assert_array_equal(b_ids, cand[order])
        np.testing.assert_allclose(b_S, S[order], rtol=1e-12)
        np.testing.assert_array_equal(a_ids, b_ids)
        np.testing.assert_array_equal(a_S, b_S)
        assert b_terms == 80 * 24 and a_terms < b_terms


def test_verify_exact_absent_and_short():
    base = np.arange(5, dtype=np.float32)[:, None]
    ids, S, _ = oracle.verify_exact(base, np.array([0], np.float32), 1.0, [3, -1, 1], 4)
    assert ids.tolist() == [1, 3, -1, -1]
    assert S[:2].tolist() == [1.0, 3.0] and np.isinf(S[2:]).all()


def test_verify_paper_worked_example():
    """K=2, kappa=2, tau=1: S values (p=1, q=0) in candidate order 5,3 | 4,1 | 6,7 | 0.5.
    R={3,5}; batch {4,1} -> R_new={1,3}, overlap 1/2 < 1; batch {6,7} ->
    R_new={1,3}, overlap 2/2 >= 1 -> stop before the last candidate."""
    vals = np.array([5, 3, 4, 1, 6, 7, 0.5], np.float32)
    base = vals[:, None]
    cand = np.arange(7, dtype=np.int32)
    ids, S, nlp, nb = oracle.verify_paper(base, np.zeros(1, np.float32), 1.0, cand, 2, 2, 1.0)
    assert ids.tolist() == [3, 1] and S.tolist() == [1.0, 3.0]
    assert nlp == 6 and nb == 2
    # a threshold above 1 never stops: the last candidate is reached
    ids, S, nlp, nb = oracle.verify_paper(base, np.zeros(1, np.float32), 1.0, cand, 2, 2, 1.5)
    assert ids.tolist() == [6, 3] and nlp == 7 and nb == 3
    # tau <= 0 stops after the first batch
    ids, S, nlp, nb = oracle.verify_paper(base, np.zeros(1, np.float32), 1.0, cand, 2, 2, 0.0)
    assert ids.tolist() == [3, 1] and nlp == 4 and nb == 1
    # ragged last batch (kappa=4 over 5 remaining -> batches of 4 and 1)
    ids, S, nlp, nb = oracle.verify_paper(base, np.zeros(1, np.float32), 1.0, cand, 2, 4, 1.5)
    assert ids.tolist() == [6, 3] and nb == 2


def test_verify_paper_never_stopping_equals_exact():
    r = rng(7)
    base = r.normal(size=(400, 16)).astype(np.float32)
    q = r.normal(size=16).astype(np.float32)
    cand = r.choice(400, size=64, replace=False).astype(np.int32)
    for p in (0.6, 1.2, 1.8):
        a, Sa, _, _ = oracle.verify_paper(base, q, p, cand, 10, 10, 1.01)
        b, Sb, _ = oracle.verify_exact(base, q, p, cand, 10)
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(Sa, Sb)


# ----------------------------------------------------------------- Algorithm 1
def test_uhnsw_full_candidate_set_equals_exact(mixture_small):
    """t = ef = N: C is every point, so both verification modes (tau > 1)
    return the exact L_p top-K of O1."""
    w, base, qs, p, g1, g2 = mixture_small
    n = len(base)
    ids_e, S_e = oracle.exact_knn(base, qs[:6], p[:6], 10)
    for mode in (0, 1):
        ids, dist, st = oracle.uhnsw_batch(g1, g2, base, qs[:6], p[:6], 10, n, t=n, tau=1.5,
                                           mode=mode)
        np.testing.assert_array_equal(ids, ids_e)
        np.testing.assert_allclose(dist, S_e ** (1 / p[:6, None].astype(np.float64)), rtol=1e-12)


def test_uhnsw_direct_p1_p2(mixture_small):
    w, base, qs, p, g1, g2 = mixture_small
    n = len(base)
    D1 = cdist(qs[:3].astype(np.float64), base.astype(np.float64), "cityblock")
    D2 = cdist(qs[:3].astype(np.float64), base.astype(np.float64), "euclidean")
    for pp, D in ((1.0, D1), (2.0, D2)):
        ids, dist, st = oracle.uhnsw_batch(g1, g2, base, qs[:3], pp, 10, n)
        for i in range(3):
            order = np.lexsort((np.arange(n), D[i]))[:10]
            np.testing.assert_array_equal(ids[i], order)
            np.testing.assert_allclose(dist[i], D[i, order], rtol=1e-12)
        assert (st[:, 1] == 0).all()      # no L_p verification


def test_uhnsw_routing_cutoff(mixture_small):
    """p <= 1.4 searches G1, p > 1.4 searches G2: a G2 whose entry point has no
    links returns only that entry point."""
    w, base, qs, p, g1, g2 = mixture_small
    n = len(base)
    dead = {"num_levels": 1, "entry_point": 7, "max_degree0": 2, "max_degree": 2, "n": n,
            "levels": [{"nodes": np.arange(n, dtype=np.int32),
                        "offsets": np.zeros(n + 1, np.int64), "nbrs": np.zeros(0, np.int32)}]}
    ids_lo, _, _ = oracle.uhnsw_query(g1, dead, base, qs[0], np.float32(1.4), 5, 32)
    ids_hi, _, _ = oracle.uhnsw_query(g1, dead, base, qs[0], np.nextafter(np.float32(1.4),
                                                                          np.float32(2)), 5, 32)
    assert (ids_lo >= 0).all()
    assert ids_hi.tolist() == [7, -1, -1, -1, -1]
    # a custom cutoff moves the boundary
    ids_c, _, _ = oracle.uhnsw_query(g1, dead, base, qs[0], np.float32(0.7), 5, 32, cutoff=0.6)
    assert ids_c.tolist() == [7, -1, -1, -1, -1]


def test_recall_definition():
    assert oracle.recall([[1, 2, 3]], [[3, 4, 1]]) == pytest.approx(2 / 3)
    assert oracle.recall([[1, 2], [5, 6]], [[1, 2], [6, 7]]) == pytest.approx(0.75)


# ----------------------------------------------------------------- U-HNSW-E (Section 4.5)
def test_base_dist_l05_pins():
    """Metric 3 is sum |d_j|^(1/2): a hand value, and scipy's Minkowski p = 0.5
    distance, which is that sum squared."""
    x = np.array([0.0, 4.0, 9.0, 2.5], np.float32)
    q = np.array([1.0, 0.0, 0.0, 2.5], np.float32)
    assert oracle.base_dist(x, q, 3) == 1.0 + 2.0 + 3.0 + 0.0
    r = rng(11)
    X = r.normal(size=(20, 24)).astype(np.float32)
    Q = r.normal(size=(3, 24)).astype(np.float32)
    D = cdist(Q.astype(np.float64), X.astype(np.float64), "minkowski", p=0.5)
    for i in range(3):
        got = [oracle.base_dist(X[j], Q[i], 3) for j in range(20)]
        np.testing.assert_allclose(got, np.sqrt(D[i]), rtol=1e-12)


@pytest.fixture(scope="module")
def mixture_e():
    w = I.WORKLOADS["mixture10k"].scaled(n=2000, nq=12)
    base = I.base_vectors(w)
    qs = I.query_vectors(w)
    g05 = oracle.hnsw_build(base, 3, w.M, w.ef_construction, I.graph_levels(w, 3))
    g1 = oracle.hnsw_build(base, 1, w.M, w.ef_construction, I.graph_levels(w, 1))
    return w, base, qs, g05, g1


def test_l05_graph_search_exact_at_full_beam(mixture_e):
    """ef >= N on the L0.5 graph gives the exact L0.5 top-t (brute force by
    scipy's Minkowski p = 0.5), and the graph keeps HNSW's degree caps."""
    w, base, qs, g05, g1 = mixture_e
    n = len(base)
    assert max(np.diff(g05["levels"][0]["offsets"]).max(), 0) <= 2 * w.M
    D = cdist(qs.astype(np.float64), base.astype(np.float64), "minkowski", p=0.5)
    for i in range(4):
        ids, dd, _ = oracle.hnsw_search(g05, base, qs[i], 3, n, 10)
        order = np.lexsort((np.arange(n), D[i]))[:10]
        np.testing.assert_array_equal(ids, order)
        np.testing.assert_allclose(dd, np.sqrt(D[i, order]), rtol=1e-12)


def test_uhnsw_e_direct_and_full_candidate_set(mixture_e):
    """U-HNSW-E (G0.5 and G1, cutoff 0.6): p = 0.5 is direct K-NN on G0.5 and
    p = 1 on G1, with no verification; with t = ef = N every p in [0.2, 1]
    returns the exact L_p top-K (O1)."""
    w, base, qs, g05, g1 = mixture_e
    n = len(base)
    E = dict(cutoff=0.6, metrics=(3, 1))
    D05 = cdist(qs[:3].astype(np.float64), base.astype(np.float64), "minkowski", p=0.5)
    D1 = cdist(qs[:3].astype(np.float64), base.astype(np.float64), "cityblock")
    for pp, D in ((0.5, D05), (1.0, D1)):
        ids, dist, st = oracle.uhnsw_batch(g05, g1, base, qs[:3], pp, 10, n, **E)
        for i in range(3):
            order = np.lexsort((np.arange(n), D[i]))[:10]
            np.testing.assert_array_equal(ids[i], order)
            np.testing.assert_allclose(dist[i], D[i, order], rtol=1e-12)
        assert (st[:, 1] == 0).all()
    pe = np.array([0.2, 0.3, 0.45, 0.6, 0.65, 0.8, 0.95, 0.55], np.float32)
    ids_e, S_e = oracle.exact_knn(base, qs[:8], pe, 10)
    ids, dist, _ = oracle.uhnsw_batch(g05, g1, base, qs[:8], pe, 10, n, t=n, tau=1.5, **E)
    np.testing.assert_array_equal(ids, ids_e)
    np.testing.assert_allclose(dist, S_e ** (1 / pe[:, None].astype(np.float64)), rtol=1e-12)


def test_uhnsw_e_routing_cutoff(mixture_e):
    """p <= 0.6 searches the first graph (G0.5), p > 0.6 the second (G1): a
    second graph whose entry point has no links returns only that entry."""
    w, base, qs, g05, g1 = mixture_e
    n = len(base)
    dead = {"num_levels": 1, "entry_point": 7, "max_degree0": 2, "max_degree": 2, "n": n,
            "levels": [{"nodes": np.arange(n, dtype=np.int32),
                        "offsets": np.zeros(n + 1, np.int64), "nbrs": np.zeros(0, np.int32)}]}
    E = dict(cutoff=0.6, metrics=(3, 1))
    lo, _, _ = oracle.uhnsw_query(g05, dead, base, qs[0], np.float32(0.6), 5, 32, **E)
    hi, _, _ = oracle.uhnsw_query(g05, dead, base, qs[0],
                                  np.nextafter(np.float32(0.6), np.float32(2)), 5, 32, **E)
    one, _, _ = oracle.uhnsw_query(g05, dead, base, qs[0], np.float32(1.0), 5, 32, **E)
    assert (lo >= 0).all()
    assert hi.tolist() == [7, -1, -1, -1, -1]
    assert one.tolist() == [7, -1, -1, -1, -1]     # p = 1 is the second graph's own metric


# ----------------------------------------------------------------- fixed-p HNSW at p = 1.5 (Section 4.3)
def test_base_dist_l15_pins():
    """Metric 4 is sum |d_j|^(3/2): a hand value, and scipy's Minkowski p = 1.5
    distance raised to 1.5."""
    x = np.array([0.0, 4.0, 9.0, 2.5], np.float32)
    q = np.array([1.0, 0.0, 0.0, 2.5], np.float32)
    assert oracle.base_dist(x, q, 4) == 1.0 + 8.0 + 27.0 + 0.0
    r = rng(12)
    X = r.normal(size=(20, 24)).astype(np.float32)
    Q = r.normal(size=(3, 24)).astype(np.float32)
    D = cdist(Q.astype(np.float64), X.astype(np.float64), "minkowski", p=1.5)
    for i in range(3):
        got = [oracle.base_dist(X[j], Q[i], 4) for j in range(20)]
        np.testing.assert_allclose(got, D[i] ** 1.5, rtol=1e-12)


def test_l15_graph_direct_queries_are_exact_at_full_beam():
    """A graph built under L1.5 answers p = 1.5 directly (no verification):
    with ef = N the answer is the exact L1.5 top-K, distances S^(1/1.5)."""
    w = I.WORKLOADS["mixture10k"].scaled(n=1500, nq=4)
    base = I.base_vectors(w)
    qs = I.query_vectors(w)
    g15 = oracle.hnsw_build(base, 4, w.M, w.ef_construction, I.graph_levels(w, 2))
    g2 = oracle.hnsw_build(base, 2, w.M, w.ef_construction, I.graph_levels(w, 2))
    n = len(base)
    D = cdist(qs.astype(np.float64), base.astype(np.float64), "minkowski", p=1.5)
    ids, dist, st = oracle.uhnsw_batch(g15, g2, base, qs, 1.5, 10, n, metrics=(4, 2))
    for i in range(len(qs)):
        order = np.lexsort((np.arange(n), D[i]))[:10]
        np.testing.assert_array_equal(ids[i], order)
        np.testing.assert_allclose(dist[i], D[i, order], rtol=1e-12)
    assert (st[:, 1] == 0).all()


# ----------------------------------------------------------------- fixed-p HNSW at any p (Section 4.3)
def _np_lp(Q, X, p):
    """S_p = sum_j |x_j - q_j|^p in float64, written out with numpy."""
    return (np.abs(Q.astype(np.float64)[:, None, :] - X.astype(np.float64)[None, :, :]) ** p).sum(-1)


def test_lp_graph_heuristic_depends_on_p_by_hand():
    """Three points inserted in order r=(0.9,-1.1), e=(2,0), q=(0,0).  From q,
    e - q = (2, 0) is sparse and e - r = (1.1, 1.1) is spread, so e is nearer
    q than r exactly when 2^p < 2 * 1.1^p, i.e. p < ln 2 / ln(2 / 1.1) ~ 1.159.
    Under L0.8 e is q's nearest and r survives the heuristic (S(r,q) = 1.998 <
    S(r,e) = 2.158), so q links to both; under L1.5 r is nearest and e is
    dropped (S(e,q) = 2.828 > S(e,r) = 2.307).  A wrong exponent (1/p, or the
    root taken inside the sum) lands on the other side of 1.159 for one of
    the two."""
    base = np.array([[0.9, -1.1], [2.0, 0.0], [0.0, 0.0]], np.float32)
    lv = np.zeros(3, np.int32)
    g = oracle.hnsw_build(base, None, M=2, ef_construction=10, levels=lv, M0=4, base_p=0.8)
    assert _lists(g, 0) == {0: [1, 2], 1: [0, 2], 2: [1, 0]}
    g = oracle.hnsw_build(base, None, M=2, ef_construction=10, levels=lv, M0=4, base_p=1.5)
    assert _lists(g, 0) == {0: [1, 2], 1: [0], 2: [0]}


def test_lp_graph_codes_are_special_cases():
    """Building under base_p 1, 2, 0.5 and 1.5 gives the same graph as the
    metric codes 1, 2, 3 and 4."""
    w = I.WORKLOADS["mixture10k"].scaled(n=600, nq=2)
    base = I.base_vectors(w)
    lv = I.graph_levels(w, 2)
    for code, bp in ((1, 1.0), (2, 2.0), (3, 0.5), (4, 1.5)):
        a = oracle.hnsw_build(base, code, w.M, w.ef_construction, lv)
        b = oracle.hnsw_build(base, None, w.M, w.ef_construction, lv, base_p=bp)
        assert a["entry_point"] == b["entry_point"]
        for la, lb in zip(a["levels"], b["levels"]):
            for key in ("nodes", "offsets", "nbrs"):
                np.testing.assert_array_equal(la[key], lb[key])


@pytest.mark.parametrize("bp", [0.8, 1.2])
def test_lp_graph_direct_and_verified_queries_at_full_beam(bp):
    """A fixed HNSW under L_bp (the same graph in both slots) answers p = bp
    directly, with distances S^(1/bp) and no L_p verification; any other p
    goes through verification of the whole candidate set.  With ef = t = N
    both are the exact top-K, against numpy brute force."""
    w = I.WORKLOADS["mixture10k"].scaled(n=1200, nq=4)
    base = I.base_vectors(w)
    qs = I.query_vectors(w)
    bp32 = float(np.float32(bp))
    g = oracle.hnsw_build(base, None, w.M, w.ef_construction, I.graph_levels(w, 2), base_p=bp)
    n = len(base)
    assert _bfs_reach(g, g["entry_point"]).all()
    for p, direct in ((bp32, True), (float(np.float32(1.37)), False)):
        S = _np_lp(qs, base, p)
        ids, dist, st = oracle.uhnsw_batch(g, g, base, qs, p, 10, n, t=n, tau=1.5,
                                           base_p=(bp, bp))
        for i in range(len(qs)):
            order = np.lexsort((np.arange(n), S[i]))[:10]
            np.testing.assert_array_equal(ids[i], order)
            np.testing.assert_allclose(dist[i], S[i, order] ** (1.0 / p), rtol=1e-12)
        assert ((st[:, 1] == 0) if direct else (st[:, 1] == n)).all()


def test_lp_graph_rejects_bad_p():
    base = np.zeros((4, 2), np.float32)
    for bp in (0.0, -1.0, 2.5):
        with pytest.raises(ValueError):
            oracle.hnsw_build(base, None, 2, 10, np.zeros(4, np.int32), base_p=bp)


def test_threaded_batch_equals_query_loop(mixture_small):
    """The multi-threaded batch driver (used to time the oracle on all host
    cores) returns what the one-query loop returns, query for query."""
    w, base, qs, p, g1, g2 = mixture_small
    ids, dist, _ = oracle.uhnsw_batch(g1, g2, base, qs, p, 10, 32)
    for threads in (1, 3, 8):
        ti, td = oracle.uhnsw_batch_threads(g1, g2, base, qs, p, 10, 32, threads)
        np.testing.assert_array_equal(ti, ids)
        np.testing.assert_array_equal(td, dist)


# ----------------------------------------------------------------- several expansions per step
def _csr1(lists, entry=0):
    n = len(lists)
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum([len(l) for l in lists])
    nbrs = np.array([v for l in lists for v in l], np.int32)
    return {"num_levels": 1, "entry_point": entry, "max_degree0": 4, "max_degree": 2, "n": n,
            "levels": [{"nodes": np.arange(n, dtype=np.int32), "offsets": offs, "nbrs": nbrs}]}


def test_wide_search_by_hand():
    """Points on a line, query at 0: E=10 (entry), A=5, B=6, C=2 (a neighbour
    of A), D=1 (a neighbour of B); ef = 2.  One expansion per step expands A
    first, C then pushes B out of W before B is expanded: W = [C, A].  Two per
    step expand A and B together, so D enters: W = [D, C]."""
    base = np.array([[10.0], [5.0], [6.0], [2.0], [1.0]], np.float32)
    g = _csr1([[1, 2], [0, 3], [0, 4], [1], [2]])
    q = np.zeros(1, np.float32)
    for width in (None, 1):
        ids, dd, nd = oracle.hnsw_search(g, base, q, 1, ef=2, t=2, width=width)
        assert ids.tolist() == [3, 1] and dd.tolist() == [2.0, 5.0] and nd == 4
    ids, dd, nd = oracle.hnsw_search(g, base, q, 1, ef=2, t=2, width=2)
    assert ids.tolist() == [4, 3] and dd.tolist() == [1.0, 2.0] and nd == 5


def test_wide_search_width1_equals_hnsw(mixture_small):
    """The width-w routine at width 1 and HNSW's SEARCH-LAYER are written
    independently; they agree id for id and distance for distance."""
    w, base, qs, p, g1, g2 = mixture_small
    for metric, g in ((1, g1), (2, g2)):
        for ef in (4, 24, 64):
            for i in range(10):
                a = oracle.hnsw_search(g, base, qs[i], metric, ef=ef, t=ef)
                b = oracle.hnsw_search(g, base, qs[i], metric, ef=ef, t=ef, width=1)
                np.testing.assert_array_equal(a[0], b[0])
                np.testing.assert_array_equal(a[1], b[1])
                assert a[2] == b[2]


@pytest.mark.parametrize("width", [2, 3, 8])
def test_wide_search_full_beam_is_exact(mixture_small, width):
    """With ef >= N every node of the connected layer 0 is reached whatever
    the width, so the first t results are the exact base-metric top-t, and
    Algorithm 1 with t = ef = N equals the exact L_p answer."""
    w, base, qs, p, g1, g2 = mixture_small
    n = len(base)
    D = cdist(qs[:3].astype(np.float64), base.astype(np.float64), "cityblock")
    for i in range(3):
        ids, dd, nd = oracle.hnsw_search(g1, base, qs[i], 1, ef=n, t=20, width=width)
        order = np.lexsort((np.arange(n), D[i]))[:20]
        np.testing.assert_array_equal(ids, order)
        assert nd >= n
    gt, _ = oracle.exact_knn(base, qs[:3], p[:3], 10)
    ids, _, _ = oracle.uhnsw_batch(g1, g2, base, qs[:3], p[:3], 10, n, t=n, width=width)
    np.testing.assert_array_equal(ids, gt)


# ----------------------------------------------------------------- construction by brute force
def _brute_build(base, levels, M, M0, metric, reach_from_entry):
    """HNSW insertion with the insertion beam replaced by brute force: at
    each level the candidates of a new node are all earlier nodes on that
    level (or, with reach_from_entry, those reachable from node 0 in the
    current single-layer graph), ranked by (distance, id); the neighbour
    heuristic keeps a candidate only if it is strictly nearer to the new node
    than to every neighbour already kept; reverse links overflowing their cap
    are re-selected by the same heuristic.  Integer data keeps every sum
    exact, so the ranking is the oracle's."""
    X = base.astype(np.float64)

    def dist(a, b):
        diff = X[a] - X[b]
        return float(np.abs(diff).sum()) if metric == 1 else float((diff * diff).sum())

    def heuristic(cand, m, b):
        out = []
        for dc, c in cand:
            if len(out) >= m:
                break
            if all(dc < dist(c, r) for r in out):
                out.append(c)
        return out

    n = len(base)
    links = [[[] for _ in range(levels[v] + 1)] for v in range(n)]
    for q in range(1, n):
        L = int(levels[:q].max())
        for lc in range(min(L, int(levels[q])), -1, -1):
            pool = [v for v in range(q) if levels[v] >= lc]
            if reach_from_entry:
                seen, stack = {0}, [0]
                while stack:
                    u = stack.pop()
                    for x in links[u][lc]:
                        if x not in seen:
                            seen.add(x)
                            stack.append(x)
                pool = [v for v in pool if v in seen]
            cand = sorted((dist(q, v), v) for v in pool)
            sel = heuristic(cand, M, q)
            links[q][lc] = sel
            cap = M0 if lc == 0 else M
            for e in sel:
                links[e][lc].append(q)
                if len(links[e][lc]) > cap:
                    c2 = sorted((dist(e, v), v) for v in links[e][lc])
                    links[e][lc] = heuristic(c2, cap, e)
    return links


@pytest.mark.parametrize("metric", [1, 2])
@pytest.mark.parametrize("seed", [0, 1])
def test_build_single_layer_equals_brute_force(metric, seed):
    """One layer, efConstruction >= N (the insertion beam reaches every node
    connected to the entry), small caps so that reverse links overflow and
    are re-selected: the construction equals the brute-force insertion."""
    r = rng(100 + seed)
    base = r.integers(0, 10, size=(90, 3)).astype(np.float32)
    lv = np.zeros(len(base), np.int32)
    g = oracle.hnsw_build(base, metric, M=3, ef_construction=200, levels=lv, M0=4)
    want = _brute_build(base, lv, 3, 4, metric, reach_from_entry=True)
    got = _lists(g, 0)
    assert got == {v: want[v][0] for v in range(len(base))}


@pytest.mark.parametrize("metric", [1, 2])
def test_build_levels_equals_brute_force(metric):
    """Several levels, caps above N (no overflow, so every level stays
    connected and the beam reaches every earlier node on it): each node's
    lists on every level equal the heuristic over all earlier nodes there."""
    r = rng(200 + metric)
    n = 70
    base = r.integers(0, 12, size=(n, 4)).astype(np.float32)
    lv = I.hnsw_levels(n, 3, 11 + metric)
    assert lv.max() >= 2
    g = oracle.hnsw_build(base, metric, M=n, ef_construction=200, levels=lv, M0=n)
    want = _brute_build(base, lv, n, n, metric, reach_from_entry=False)
    for l in range(g["num_levels"]):
        got = _lists(g, l)
        assert got == {v: want[v][l] for v in range(n) if lv[v] >= l}, f"level {l}"


# ----------------------------------------------------------------- precision form (rounded rows)
def _f16_rows(x):
    return x.astype(np.float16).astype(np.float32)


def test_trav_equal_to_base_is_the_plain_query(mixture_small):
    """With the traversal rows equal to the FP32 rows, the precision form is
    Algorithm 1 itself: same ids and distances for general p, p = 1 and
    p = 2 (the direct queries' beam re-rank keeps the beam's order), at
    widths 1 and 2, in both verification modes."""
    w, base, qs, p, g1, g2 = mixture_small
    ps = np.concatenate([p[:6], [1.0, 2.0]]).astype(np.float32)
    for width in (1, 2):
        for mode in (0, 1):
            for i, pp in enumerate(ps):
                a = oracle.uhnsw_query(g1, g2, base, qs[i], float(pp), 10, 40, mode=mode,
                                       width=width)
                b = oracle.uhnsw_query_trav(g1, g2, base, base, qs[i], float(pp), 10, 40,
                                            mode=mode, width=width)
                np.testing.assert_array_equal(a[0], b[0])
                np.testing.assert_allclose(a[1], b[1], rtol=1e-12)
                assert a[2][0] == b[3][0]                 # same N_b


def test_trav_full_beam_ranks_by_rounded_rows(mixture_small):
    """ef >= N on a connected layer 0: the candidate list is the exact top-t
    under the base metric of the ROUNDED rows (brute force on them), and the
    answer is the exact L_p top-K over that list on the FP32 rows; a direct
    p = 1 query returns the FP32 L1 top-K of its whole (rounded-row) beam."""
    w, base, qs, p, g1, g2 = mixture_small
    trav = _f16_rows(base)
    assert (trav != base).mean() > 0.5
    n, t = len(base), 25
    for i in range(4):
        pp = float(p[i])
        metric, g = ((1, "cityblock") if pp <= 1.4 else (2, "sqeuclidean"))
        D = cdist(qs[i:i + 1].astype(np.float64), trav.astype(np.float64), g)[0]
        top_t = np.lexsort((np.arange(n), D))[:t]
        ids, dist, cand, st = oracle.uhnsw_query_trav(g1, g2, base, trav, qs[i], pp, 10, n, t=t)
        np.testing.assert_array_equal(cand[:t], top_t)
        S = (np.abs(base[top_t].astype(np.float64) - qs[i].astype(np.float64)) ** pp).sum(1)
        order = top_t[np.lexsort((top_t, S))][:10]
        np.testing.assert_array_equal(ids, order)
        np.testing.assert_allclose(dist, np.sort(S)[:10] ** (1 / pp), rtol=1e-12)
    D1 = cdist(qs[:1].astype(np.float64), base.astype(np.float64), "cityblock")[0]
    ids, dist, cand, st = oracle.uhnsw_query_trav(g1, g2, base, trav, qs[0], 1.0, 10, n)
    order = np.lexsort((np.arange(n), D1))[:10]
    np.testing.assert_array_equal(ids, order)
    np.testing.assert_allclose(dist, D1[order], rtol=1e-12)


def test_near_tie_counter_sees_equal_distances():
    """Two points at the same distance from the query (mirror images) make
    the search compare equal values: counted at any tolerance; points far
    apart in distance are not counted at a small tolerance; the count never
    falls as the tolerance grows."""
    base = np.array([[0.0], [10.0], [-3.0], [3.0], [7.5], [-8.0]], np.float32)
    g = oracle.hnsw_build(base, 1, M=4, ef_construction=10, levels=np.zeros(6, np.int32), M0=8)
    q = np.array([0.0], np.float32)
    counts = []
    for tol in (1e-12, 1e-6, 0.3, 1.0):
        _, _, _, st = oracle.uhnsw_query_trav(g, g, base, base, q, 1.0, 3, 6, tie_tol=tol)
        counts.append(int(st[3]))
    assert counts[0] >= 1                      # |-3| == |3|
    assert counts == sorted(counts)
    base2 = np.array([[0.0], [10.0], [-3.0], [3.5], [7.5], [-8.0]], np.float32)
    g2 = oracle.hnsw_build(base2, 1, M=4, ef_construction=10, levels=np.zeros(6, np.int32), M0=8)
    _, _, _, st = oracle.uhnsw_query_trav(g2, g2, base2, base2, q, 1.0, 3, 6, tie_tol=1e-6)
    assert st[3] == 0


def _round_mantissa(x, keep):
    """FP32 values rounded (to nearest, ties to even) to `keep` mantissa bits."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    drop = 23 - keep
    r = ((u + (1 << (drop - 1)) - 1 + ((u >> drop) & 1)) >> drop) << drop
    return r.astype(np.uint32).view(np.float32)


def test_tie_free_searches_survive_perturbation(mixture_small):
    """The certificate behind the float-data parity rule: if the search on
    one copy of the rows made no comparison within tol (relative), a second
    copy whose every base distance differs from the first by less than tol / 2
    (relative) gives the same candidate list.  The second copies are the FP32
    rows rounded to 12 and 14 mantissa bits; tol is just over twice their
    largest relative distance difference from the FP32 rows (brute force
    over every node).  Every query whose candidate lists differ must have
    counted a near-tie, some lists do differ, and some searches are
    tie-free."""
    w, base, qs, p, g1, g2 = mixture_small
    nq = 20
    flagged = diverged = total = 0
    for keep in (12, 14):
        trav = _round_mantissa(base, keep)
        rel = 0.0
        for name in ("cityblock", "sqeuclidean"):
            A = cdist(qs[:nq].astype(np.float64), base.astype(np.float64), name)
            B = cdist(qs[:nq].astype(np.float64), trav.astype(np.float64), name)
            rel = max(rel, float((np.abs(A - B) / np.maximum(np.maximum(A, B), 1e-300)).max()))
        tol = 2.0 * rel * 1.01
        for i in range(nq):
            for width in (1, 2):
                a = oracle.uhnsw_query_trav(g1, g2, base, base, qs[i], float(p[i]), 10, 32,
                                            width=width, tie_tol=tol)
                b = oracle.uhnsw_query_trav(g1, g2, base, trav, qs[i], float(p[i]), 10, 32,
                                            width=width, tie_tol=tol)
                if a[3][3] == 0:
                    np.testing.assert_array_equal(a[2], b[2])
                flagged += int(a[3][3] > 0)
                diverged += int(not np.array_equal(a[2], b[2]))
                total += 1
    assert diverged >= 1 and flagged < total
