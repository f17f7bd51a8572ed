"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Verification: ids identical to the oracle's exhaustive top-K over the same
candidate set except near-ties within 1e-5 relative; distances within 2e-5
relative.  Deterministic search (one expansion per step): the beam equals the
oracle's HNSW search on the same CSR id for id (integer / grid data make the
FP32 base distances exact).  Sizes span several tiles and ragged tails."""
import numpy as np
import pytest

import oracle
from paper_2605_02030_gb300 import inputs as I

from helpers import check_topk, oracle_graphs, workload_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    import paper_2605_02030_gb300 as pkg
    pkg.build()
    from paper_2605_02030_gb300 import uhnsw
    uhnsw.load_library()
    return uhnsw


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ------------------------------------------------------------------ verification
@pytest.fixture(scope="module")
def mix_small():
    return workload_arrays("mixture10k", 2000, 24)


@pytest.fixture(scope="module")
def sift_small():
    return workload_arrays("sift1m", 3000, 24)


@pytest.mark.parametrize("which", ["mix", "sift"])
@pytest.mark.parametrize("k,t", [(1, 17), (10, 64), (10, 301), (100, 300)])
def test_verify_exact_matches_oracle(U, mix_small, sift_small, which, k, t):
    w, base, qs, p, _, _ = mix_small if which == "mix" else sift_small
    nq = len(qs)
    pv = p.copy()
    pv[:6] = [0.5, 1.5, 1.0, 2.0, 0.51, 1.93]      # the SFU-free / one-sqrt cases
    cand = I.random_candidates(len(base), nq, t, seed=11 + t, missing_frac=0.2)
    idx = U.Index(base, None, oracle_graphs("mixture10k", 2000, 24)[1] if which == "mix" else
                  oracle_graphs("sift1m", 3000, 24, M=8, ef_construction=40)[1])
    ids, dist, st = idx.verify(dev(qs), dev(pv), dev(cand), k, stats=True)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    for i in range(nq):
        rid, rS, _ = oracle.verify_exact(base, qs[i], pv[i], cand[i], k)
        check_topk(base, qs[i], pv[i], ids[i], dist[i], rid, k, f"q{i}")
        assert st[i, 5] == 0
        assert st[i, 1] == (cand[i] >= 0).sum()       # every valid candidate started
    # the partial-sum drop (checked every 32 dimensions) skips terms once the
    # k-th best is known
    if t >= 64 and w.d >= 64:
        assert st[:, 2].sum() < ((cand >= 0).sum(axis=1) * w.d).sum()
    idx.close()


@pytest.mark.parametrize("tau", [-1.0, 0.5, 0.92, 1.0, 1.5])
@pytest.mark.parametrize("kappa", [0, 3, 25])
def test_verify_paper_mode_matches_oracle(U, sift_small, tau, kappa):
    w, base, qs, p, _, _ = sift_small
    k, t = 10, 120
    nq = len(qs)
    cand = I.random_candidates(len(base), nq, t, seed=5)
    # candidate order matters in Algorithm 1: sort by L1 like a real C
    for i in range(nq):
        dl1 = np.abs(base[cand[i]] - qs[i]).sum(1)
        cand[i] = cand[i][np.lexsort((cand[i], dl1))]
    idx = U.Index(base, None, oracle_graphs("sift1m", 3000, 24, M=8, ef_construction=40)[1])
    ids, dist, st = idx.verify(dev(qs), dev(p), dev(cand), k, mode="paper", kappa=kappa, tau=tau,
                               stats=True)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    same_np = 0
    for i in range(nq):
        rid, rS, nlp, nb = oracle.verify_paper(base, qs[i], p[i], cand[i], k, kappa or k, tau)
        ties = check_topk(base, qs[i], p[i], ids[i], dist[i], rid, k, f"q{i}")
        same_np += int(st[i, 1] == nlp)
        if ties == 0:
            assert st[i, 1] == nlp, f"q{i}: {st[i, 1]} L_p candidates vs oracle {nlp}"
    assert same_np >= nq - 1
    idx.close()


def test_verify_degenerate(U, sift_small):
    w, base, qs, p, _, _ = sift_small
    idx = U.Index(base, None, oracle_graphs("sift1m", 3000, 24, M=8, ef_construction=40)[1])
    cand = np.full((3, 5), -1, np.int32)
    cand[1, 2] = 7
    pv = np.array([0.7, 1.2, 2.0], np.float32)
    ids, dist, _ = idx.verify(dev(qs[:3]), dev(pv), dev(cand), 4)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    assert (ids[0] == -1).all() and np.isinf(dist[0]).all()
    assert ids[1].tolist() == [7, -1, -1, -1]
    assert dist[1, 0] == pytest.approx(oracle.lp_sum(base[7], qs[1], 1.2) ** (1 / np.float32(1.2)),
                                       rel=2e-5)
    # invalid p -> that query alone is padded and flagged
    pv = np.array([0.0, 2.5, 1.0], np.float32)
    cand = np.tile(np.arange(5, dtype=np.int32), (3, 1))
    ids, dist, st = idx.verify(dev(qs[:3]), dev(pv), dev(cand), 2, stats=True)
    st = st.cpu().numpy()
    assert st[0, 5] == -1 and st[1, 5] == -1 and st[2, 5] == 0
    assert (ids.cpu().numpy()[:2] == -1).all()
    # nq = 0 is a no-op
    e = torch.empty((0, 128), device="cuda")
    idx.verify(e, torch.empty(0, device="cuda"), torch.empty((0, 5), dtype=torch.int32, device="cuda"), 2)
    idx.close()


# ------------------------------------------------------------------ exact k-NN
@pytest.mark.parametrize("which,k", [("mix", 1), ("mix", 10), ("sift", 10), ("sift", 100)])
def test_exact_knn_matches_oracle(U, mix_small, sift_small, which, k):
    w, base, qs, p, _, _ = mix_small if which == "mix" else sift_small
    pv = p.copy()
    pv[:2] = [1.0, 2.0]
    idx = U.Index(base, *(oracle_graphs("mixture10k", 2000, 24) if which == "mix" else
                          oracle_graphs("sift1m", 3000, 24, M=8, ef_construction=40)))
    ids, dist = idx.exact(dev(qs), dev(pv), k)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    rid, rS = oracle.exact_knn(base, qs, pv, k)
    for i in range(len(qs)):
        check_topk(base, qs[i], pv[i], ids[i], dist[i], rid[i], k, f"q{i}")
    idx.close()


# ------------------------------------------------------------------ search
CASES = {
    # name: (workload, n, nq, grid, kw)
    "mixture_grid": ("mixture10k", 4000, 40, 1 / 16, {}),
    "sift": ("sift1m", 6000, 40, 0.0, dict(M=12, ef_construction=80)),
}


@pytest.fixture(params=[32, 128], ids=["warp", "block"])
def qt(request):
    """threads per query: 32 = warp-per-query kernel, 128 = block-per-query kernel"""
    return request.param


@pytest.fixture(scope="module", params=list(CASES))
def search_case(request, U):
    name, n, nq, grid, kw = CASES[request.param]
    w, base, qs, p, k, ef = workload_arrays(name, n, nq, grid, **kw)
    g1, g2 = oracle_graphs(name, n, nq, grid, **kw)
    return request.param, w, base, qs, p, g1, g2


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("ef", [16, 50, 128])
def test_deterministic_beam_equals_oracle_search(U, search_case, dtype, ef, qt):
    """p = 1 and p = 2 return the first k beam entries directly: with k = ef
    this is the whole beam, which must equal the oracle's SEARCH-LAYER result
    on the same graph id for id (base distances exact on this data)."""
    cname, w, base, qs, p, g1, g2 = search_case
    if dtype == "bf16" and cname == "mixture_grid":
        pytest.skip("grid values are not exact in BF16")
    idx = U.Index(base, g1, g2, traverse_dtype=dtype)
    nq = len(qs)
    for pp, metric, g in ((1.0, 1, g1), (2.0, 2, g2)):
        pv = np.full(nq, pp, np.float32)
        ids, dist, st = idx.search(dev(qs), dev(pv), k=ef, ef=ef, stats=True, query_threads=qt)
        ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
        for i in range(nq):
            rid, rd, _ = oracle.hnsw_search(g, base, qs[i], metric, ef, ef)
            np.testing.assert_array_equal(ids[i], rid, err_msg=f"{cname} {dtype} p={pp} q{i}")
            want = rd if metric == 1 else np.sqrt(rd)
            np.testing.assert_allclose(dist[i][rid >= 0], want[rid >= 0], rtol=1e-6)
        assert (st[:, 6] == metric).all() and (st[:, 5] == 0).all()
    idx.close()


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_uhnsw_query_matches_oracle(U, search_case, mode, qt):
    """Algorithm 1 end to end (routing, KnnSearch, verification) against the
    oracle on the same graphs, per-query p (including p = 1, 2 and the
    1.4 cutoff on both sides), k = 10, ef = 48, t = ef."""
    cname, w, base, qs, p, g1, g2 = search_case
    nq = len(qs)
    pv = p.copy()
    pv[:5] = [1.0, 2.0, 1.4, np.nextafter(np.float32(1.4), np.float32(2)), 0.5]
    idx = U.Index(base, g1, g2)
    ids, dist, st = idx.search(dev(qs), dev(pv), k=10, ef=48, mode=mode, stats=True,
                               query_threads=qt)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    for i in range(nq):
        rid, rd, rst = oracle.uhnsw_query(g1, g2, base, qs[i], pv[i], 10, 48,
                                          mode=0 if mode == "exact" else 1)
        check_topk(base, qs[i], pv[i], ids[i], dist[i], rid, 10, f"{cname} q{i} p={pv[i]}")
        exp_graph = 1 if pv[i] == 1.0 else 2 if pv[i] == 2.0 else (1 if pv[i] <= np.float32(1.4) else 2)
        assert st[i, 6] == exp_graph
    idx.close()


def test_search_per_query_k_ef_and_padding(U, search_case, qt):
    cname, w, base, qs, p, g1, g2 = search_case
    nq = len(qs)
    rng = np.random.default_rng(3)
    k = rng.integers(1, 21, nq).astype(np.int32)
    ef = np.maximum(rng.integers(8, 90, nq), 1).astype(np.int32)
    idx = U.Index(base, g1, g2)
    ids, dist, _ = idx.search(dev(qs), dev(p), k=dev(k), ef=dev(ef), k_max=24, ef_max=128,
                              query_threads=qt)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    for i in range(nq):
        rid, rd, _ = oracle.uhnsw_query(g1, g2, base, qs[i], p[i], int(k[i]), int(ef[i]))
        check_topk(base, qs[i], p[i], ids[i], dist[i], rid, int(k[i]), f"q{i}")
        assert (ids[i, k[i]:] == -1).all() and np.isinf(dist[i, k[i]:]).all()
    idx.close()


def test_search_forms_agree_bitwise(U, search_case, qt):
    """Plain launch, persistent launch, CUDA-graph replay, host-buffer call and
    each query alone vs in the batch: identical results (deterministic mode)."""
    cname, w, base, qs, p, g1, g2 = search_case
    idx = U.Index(base, g1, g2, traverse_dtype="f16")
    q, pp = dev(qs), dev(p)
    a_ids, a_d, _ = idx.search(q, pp, k=10, ef=40, query_threads=qt)
    b_ids, b_d, _ = idx.search(q, pp, k=10, ef=40, persistent=True, query_threads=qt)
    c_ids, c_d, _ = idx.search(q, pp, k=10, ef=40, persistent=True, use_graph=True,
                               query_threads=qt)
    c2_ids, c2_d, _ = idx.search(q, pp, k=10, ef=40, persistent=True, use_graph=True,
                                 out=(c_ids, c_d), query_threads=qt)
    h_ids, h_d = idx.search_host(qs, p, k=10, ef=40, query_threads=qt)
    torch.cuda.synchronize()
    for x, y in ((b_ids, b_d), (c_ids, c_d), (c2_ids, c2_d)):
        assert torch.equal(a_ids, x) and torch.equal(a_d, y)
    np.testing.assert_array_equal(a_ids.cpu().numpy(), h_ids)
    np.testing.assert_array_equal(a_d.cpu().numpy(), h_d)
    for i in (0, 7, len(qs) - 1):
        s_ids, s_d, _ = idx.search(q[i:i + 1], pp[i:i + 1], k=10, ef=40, query_threads=qt)
        assert torch.equal(s_ids[0], a_ids[i]) and torch.equal(s_d[0], a_d[i])
    idx.close()


def test_wide_search_recall_and_validity(U, search_case, qt):
    """Several expansions per step (not HNSW's sequential order): results stay
    valid and recall against the exact answer stays high."""
    cname, w, base, qs, p, g1, g2 = search_case
    idx = U.Index(base, g1, g2)
    gt, _ = oracle.exact_knn(base, qs, p, 10)
    for width in (2, 4):
        ids, dist, _ = idx.search(dev(qs), dev(p), k=10, ef=64, width=width, query_threads=qt)
        ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
        for i in range(len(qs)):
            got = ids[i][ids[i] >= 0]
            assert len(set(got.tolist())) == len(got)
            for j, v in enumerate(got):
                exp = oracle.lp_sum(base[v], qs[i], float(p[i])) ** (1 / float(p[i]))
                assert abs(dist[i, j] - exp) <= 2e-5 * exp
        assert oracle.recall(ids, gt) >= 0.9
    idx.close()


def test_search_invalid_queries_and_edges(U, search_case, qt):
    cname, w, base, qs, p, g1, g2 = search_case
    idx = U.Index(base, g1, None)
    pv = np.array([0.8, -1.0, 1.9, np.nan], np.float32)   # 1.9 routes to the missing G2
    ids, dist, st = idx.search(dev(qs[:4]), dev(pv), k=5, ef=20, stats=True, query_threads=qt)
    st = st.cpu().numpy()
    assert st[0, 5] == 0 and (st[1:, 5] == -1).all()
    assert (ids.cpu().numpy()[1:] == -1).all()
    # k above ef: the beam grows to k
    ids, dist, _ = idx.search(dev(qs[:2]), dev(np.array([0.9, 0.9], np.float32)), k=30, ef=8,
                              query_threads=qt)
    assert (ids.cpu().numpy() >= 0).all()
    # empty batch
    idx.search(torch.empty((0, w.d), device="cuda"), torch.empty(0, device="cuda"), k=5, ef=20,
               query_threads=qt)
    torch.cuda.synchronize()
    assert idx.device_status() == 0
    idx.close()


def test_tiny_graph_fewer_points_than_k(U):
    base = np.array([[0.0] * 8, [1.0] * 8, [3.0] * 8], np.float32)
    g = oracle.hnsw_build(base, 1, 2, 4, np.zeros(3, np.int32))
    g2 = oracle.hnsw_build(base, 2, 2, 4, np.zeros(3, np.int32))
    idx = U.Index(base, g, g2)
    q = np.array([[0.9] * 8], np.float32)
    ids, dist, _ = idx.search(dev(q), dev(np.array([0.7], np.float32)), k=5, ef=8)
    assert ids.cpu().numpy().tolist() == [[1, 0, 2, -1, -1]]
    assert np.isinf(dist.cpu().numpy()[0, 3:]).all()
    idx.close()


@pytest.mark.parametrize("dtype,persistent", [("f32", False), ("f16", True)])
def test_large_batch_replicas_agree(U, search_case, dtype, persistent, qt):
    """Thousands of resident blocks (many per SM) with a small beam, so the
    visited table resets every few steps: each replicated query must return
    exactly the result it returns alone, and the device error word stays 0."""
    cname, w, base, qs, p, g1, g2 = search_case
    reps = 160
    qbig = np.tile(qs, (reps, 1))
    pbig = np.tile(p, reps)
    idx = U.Index(base, g1, g2, traverse_dtype=dtype)
    for ef in (16, 48):
        ids, dist, st = idx.search(dev(qbig), dev(pbig), k=10, ef=ef, persistent=persistent,
                                   stats=True, query_threads=qt)
        one, one_d, _ = idx.search(dev(qs), dev(p), k=10, ef=ef, query_threads=qt)
        torch.cuda.synchronize()
        assert idx.device_status() == 0
        ids = ids.cpu().numpy().reshape(reps, len(qs), 10)
        dist = dist.cpu().numpy().reshape(reps, len(qs), 10)
        one, one_d = one.cpu().numpy(), one_d.cpu().numpy()
        assert (st.cpu().numpy()[:, 5] == 0).all()
        for r in range(reps):
            np.testing.assert_array_equal(ids[r], one)
            np.testing.assert_array_equal(dist[r], one_d)
    idx.close()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_warp_and_block_kernels_agree(U, search_case, dtype):
    """The warp-per-query and block-per-query kernels run the same algorithm:
    on exact data (integer / grid) they return identical ids and distances."""
    cname, w, base, qs, p, g1, g2 = search_case
    idx = U.Index(base, g1, g2, traverse_dtype=dtype)
    for mode in ("exact", "paper"):
        a = idx.search(dev(qs), dev(p), k=10, ef=40, mode=mode, query_threads=32)
        b = idx.search(dev(qs), dev(p), k=10, ef=40, mode=mode, query_threads=128)
        torch.cuda.synchronize()
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    idx.close()


def test_autotune_picks_a_valid_configuration(U, search_case, tmp_path):
    """The autotuner times the compiled launch configurations, records the
    fastest for the bucket, and later searches with query_threads == 0 use it:
    same ids and distances as the explicit configuration (exact data)."""
    cname, w, base, qs, p, g1, g2 = search_case
    idx = U.Index(base, g1, g2, traverse_dtype="f16")
    q, pp = dev(qs), dev(p)
    best, ms = idx.autotune(q, pp, 10, 40)
    assert best["query_threads"] in (32, 128) and ms > 0
    if best["query_threads"] == 32:
        assert best["team_lanes"] in (4, 8, 16, 32) and best["stage_bytes"] % (4 * w.d) == 0
    # the drop-test interval is searched for the warp kernel only (the block
    # kernel tests after every group)
    assert best["verify_groups"] in ((1, 2, 4) if best["query_threads"] == 32 else (0,))
    assert best["hash_bits"] >= 0
    tuned = idx.search(q, pp, k=10, ef=40)
    explicit = idx.search(q, pp, k=10, ef=40, **best)
    torch.cuda.synchronize()
    assert torch.equal(tuned[0], explicit[0]) and torch.equal(tuned[1], explicit[1])
    path = str(tmp_path / "tuned.txt")
    idx.autotune_save(path)
    line = open(path).read().split()
    assert len(line) == 9 and int(line[1]) == w.d and int(line[4]) == best["query_threads"]
    assert int(line[7]) == best["hash_bits"] and int(line[8]) == best["verify_groups"]
    idx2 = U.Index(base, g1, g2, traverse_dtype="f16")
    idx2.autotune_load(path)
    again = idx2.search(q, pp, k=10, ef=40)
    torch.cuda.synchronize()
    assert torch.equal(again[0], tuned[0]) and torch.equal(again[1], tuned[1])
    idx.close()
    idx2.close()


def test_table_size_and_drop_interval_change_no_result(U, search_case, qt):
    """The autotuner's visited-table size, drop-test interval and staged
    verification rows leave every sum and decision of the search unchanged:
    any allowed table size (from the smallest that holds a beam plus one
    step of candidates), a drop test every 1 to 5 verification groups and 4
    or 16 staged rows return the default call's ids and distances bit for
    bit, in both verification modes, and so does the verification-only entry
    point.  A table below the minimum is refused."""
    import math

    cname, w, base, qs, p, g1, g2 = search_case
    idx = U.Index(base, g1, g2, traverse_dtype="f32")
    q, pp = dev(qs), dev(p)
    ef, width = 40, 2
    m0 = max(g1["max_degree0"], g2["max_degree0"])
    lo = math.ceil(math.log2(2 * (ef + width * m0)))
    for mode in ("exact", "paper"):
        ref = idx.search(q, pp, k=10, ef=ef, width=width, mode=mode, query_threads=qt)
        for hb in (lo, lo + 1, lo + 2):
            for vg in (1, 2, 3, 5):
                got = idx.search(q, pp, k=10, ef=ef, width=width, mode=mode, query_threads=qt,
                                 hash_bits=hb, verify_groups=vg)
                torch.cuda.synchronize()
                assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]), (mode, hb, vg)
        if qt == 32:
            # the staged verification rows at once (default: what the table's bytes hold)
            for rows in (4, 16):
                got = idx.search(q, pp, k=10, ef=ef, width=width, mode=mode, query_threads=qt,
                                 stage_bytes=rows * 4 * base.shape[1])
                torch.cuda.synchronize()
                assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]), (mode, rows)
    with pytest.raises(U.UHNSWError):
        idx.search(q, pp, k=10, ef=ef, width=width, query_threads=qt, hash_bits=lo - 1)
    cand = torch.from_numpy(np.stack([np.random.default_rng(i).choice(len(base), 60, replace=False)
                                      for i in range(len(qs))]).astype(np.int32)).cuda()
    vref = idx.verify(q, pp, cand, 10)
    for vg in (2, 4, 16):
        got = idx.verify(q, pp, cand, 10, verify_groups=vg)
        torch.cuda.synchronize()
        assert torch.equal(got[0], vref[0]) and torch.equal(got[1], vref[1])
    assert idx.device_status() == 0
    idx.close()


def test_bucketed_persistent_queue_matches_plain(U, search_case, qt):
    """Per-query ef across several beam buckets: the bucketed persistent launch
    (one launch per bucket) returns what one plain launch returns."""
    cname, w, base, qs, p, g1, g2 = search_case
    rng = np.random.default_rng(9)
    nq = len(qs)
    k = rng.choice([1, 10, 20], size=nq).astype(np.int32)
    ef = rng.choice([16, 40, 100, 200, 300], size=nq).astype(np.int32)
    idx = U.Index(base, g1, g2, traverse_dtype="f16")
    a = idx.search(dev(qs), dev(p), k=dev(k), ef=dev(ef), k_max=20, ef_max=300,
                   query_threads=qt, stats=True)
    b = idx.search(dev(qs), dev(p), k=dev(k), ef=dev(ef), k_max=20, ef_max=300,
                   query_threads=qt, persistent=True, stats=True)
    c = idx.search(dev(qs), dev(p), k=dev(k), ef=dev(ef), k_max=20, ef_max=300,
                   query_threads=qt, persistent=True, use_graph=True)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])
    assert (b[2].cpu().numpy()[:, 5] == 0).all()
    assert idx.device_status() == 0
    idx.close()


def test_queue_route_order_and_kernel_events(U, search_case, qt):
    """The persistent queue ordered by (beam bucket, route) returns what the
    plain launch returns for a mix of routes (G1 / G2, direct p, p = 0.5 and
    1.5, general p), and the kernel_events option brackets the search kernels
    without changing any result, plain and under CUDA-graph replay."""
    cname, w, base, qs, p, g1, g2 = search_case
    nq = len(qs)
    pr = np.resize(np.array([1.0, 2.0, 0.5, 1.5, 0.7, 1.3, 1.8, 1.4], np.float32), nq)
    np.random.default_rng(4).shuffle(pr)
    idx = U.Index(base, g1, g2, traverse_dtype="f16")
    a = idx.search(dev(qs), dev(pr), k=10, ef=32, query_threads=qt, stats=True)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for e in ev:
        e.record()
    for graph in (False, True):
        for _ in range(2):
            b = idx.search(dev(qs), dev(pr), k=10, ef=32, query_threads=qt, persistent=True,
                           use_graph=graph, kernel_events=ev)
            torch.cuda.synchronize()
            assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
            assert ev[0].elapsed_time(ev[1]) > 0.0
    st = a[2].cpu().numpy()
    assert (st[:, 5] == 0).all()
    assert set(np.unique(st[:, 6]).tolist()) == {1, 2}
    bad = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    if int(bad[0].cuda_event) == 0:                  # torch creates events at first record
        with pytest.raises(ValueError):
            idx.search(dev(qs), dev(pr), k=10, ef=32, kernel_events=bad)
    assert idx.device_status() == 0
    idx.close()


def test_large_beam_buckets_fall_back_to_the_block_kernel(U):
    """A beam bucket too large for four warp-kernel queries per block runs the
    block kernel when query_threads is left to the library, and returns what
    the block kernel alone returns; forcing the warp kernel fails cleanly."""
    w, base, qs, p, _, _ = workload_arrays("mixture10k", 3000, 40, 1 / 16)
    g1, g2 = oracle_graphs("mixture10k", 3000, 40, 1 / 16)
    idx = U.Index(base, g1, g2, traverse_dtype="f32")
    ef = np.where(np.arange(len(qs)) % 2 == 0, 32, 500).astype(np.int32)
    # 384 staged rows (48 KB per query, sharing its region with the visited
    # table): the ef <= 64 bucket fits four warp queries per block (204 KB),
    # the ef 512 bucket does not (232,704 B > 227 KB)
    kw = dict(k=10, ef=dev(ef), k_max=10, ef_max=512, stage_bytes=49152)
    a = idx.search(dev(qs), dev(p), persistent=True, **kw)
    b = idx.search(dev(qs), dev(p), query_threads=128, **kw)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    with pytest.raises(U.UHNSWError):
        idx.search(dev(qs), dev(p), query_threads=32, **kw)
    assert idx.device_status() == 0
    idx.close()
