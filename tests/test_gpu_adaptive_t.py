"""Per-query t and tau (the t / tau trade-off of Section 3.2 as a per-query
knob) and the idealized-recall curves behind the choice of t, on the GPU.

- The curves equal their definition applied to the oracle's exact answers:
  counts[t-1] = |exact L_p top-K & exact base-metric top-t|.  Integer data
  and p = 2 against the L1 graph of a U-HNSW-E index make both exact orders
  FP32-exact.
- A batch with per-query t / tau returns, for every query, what a batch with
  that query's t / tau as the scalar option returns (bit for bit), in the
  plain and the persistent (beam-bucketed) forms."""
import numpy as np
import pytest

import oracle
from paper_2605_02030_gb300 import inputs as I

from helpers import oracle_graphs, workload_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
def sift_case():
    w, base, qs, p, _, _ = workload_arrays("sift1m", 3000, 48, M=8, ef_construction=40)
    g1, g2 = oracle_graphs("sift1m", 3000, 48, M=8, ef_construction=40)
    return w, base, qs, p, g1, g2


def test_idealized_recall_matches_definition(U, sift_case):
    w, base, qs, p, g1, g2 = sift_case
    nq, K, T = len(qs), 10, 64
    # an index whose graphs are under L0.5 and L1 routes p = 2 to the L1 graph:
    # exact L2 top-K against exact L1 top-t, both exact sums on integer data
    g05 = oracle.hnsw_build(base, 3, 8, 30, I.hnsw_levels(len(base), 8, 5))
    idx = U.Index(base, g05, g1, metrics=U.U_HNSW_E)
    pv = np.full(nq, 2.0, np.float32)
    pv[::3] = 1.0                     # the L1 graph's own p: the curve reaches K at t = K
    counts = idx.idealized_recall(dev(qs), dev(pv), K, T, cutoff=0.6).cpu().numpy()
    topk, _ = oracle.exact_knn(base, qs, pv, K)
    topt, _ = oracle.exact_knn(base, qs, np.ones(nq, np.float32), T)
    for i in range(nq):
        want = [len(set(topk[i].tolist()) & set(topt[i, :t].tolist())) for t in range(1, T + 1)]
        np.testing.assert_array_equal(counts[i], want, err_msg=f"query {i} p={pv[i]}")
        if pv[i] == 1.0:
            assert counts[i, K - 1] == K
    assert (np.diff(counts, axis=1) >= 0).all() and (counts[:, -1] <= K).all()
    idx.close()


@pytest.mark.parametrize("mode", ["exact", "paper"])
@pytest.mark.parametrize("persistent", [False, True])
def test_per_query_t_and_tau_equal_scalar_calls(U, sift_case, mode, persistent):
    w, base, qs, p, g1, g2 = sift_case
    nq = len(qs)
    idx = U.Index(base, g1, g2, traverse_dtype="f16")
    choices_t = np.array([0, 10, 24, 60, 130], np.int32)       # 0 = ef
    choices_tau = np.array([0.0, 0.8, 1.5, -1.0], np.float32)  # 0 = 0.92
    r = np.random.default_rng(5)
    tq = choices_t[r.integers(0, len(choices_t), nq)]
    tauq = choices_tau[r.integers(0, len(choices_tau), nq)]
    kw = dict(k=10, ef=32, mode=mode, ef_max=160, persistent=persistent)
    ids, dist, st = idx.search(dev(qs), dev(p), t=dev(tq), tau=dev(tauq), stats=True, **kw)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    assert (st[:, 5] == 0).all()
    for tv in choices_t:
        for tauv in choices_tau:
            sel = np.nonzero((tq == tv) & (tauq == tauv))[0]
            if len(sel) == 0:
                continue
            a, b, _ = idx.search(dev(qs[sel]), dev(p[sel]), t=int(tv), tau=float(tauv),
                                 **dict(kw, ef_max=0))
            np.testing.assert_array_equal(ids[sel], a.cpu().numpy(), err_msg=f"t={tv} tau={tauv}")
            np.testing.assert_array_equal(dist[sel], b.cpu().numpy())
    # the host-buffer entry point takes the same per-query arrays from host memory
    hi, hd = idx.search_host(qs, p, t=tq, tau=tauq, **kw)
    np.testing.assert_array_equal(hi, ids)
    np.testing.assert_array_equal(hd, dist)
    assert idx.device_status() == 0
    idx.close()


def test_planned_t_reaches_the_search(U, sift_case):
    """End to end: curves on the queries, a t per p bin, then a search with
    those t.  A higher target never plans a smaller t; each non-direct query
    verifies exactly its planned t candidates (exact mode starts an L_p sum
    for every candidate: N_p = t); direct queries (p = 1, 2) verify none.
    The plan assumes the true base-metric top-t, which the beam only
    approximates, so recall itself is a bench figure, not asserted here."""
    w, base, qs, p, g1, g2 = sift_case
    idx = U.Index(base, g1, g2, traverse_dtype="f16")
    counts = idx.idealized_recall(dev(qs), dev(p), 10, 128).cpu().numpy()
    lo = U.plan_t(counts, p, 10, 0.9)
    hi = U.plan_t(counts, p, 10, 0.99)
    assert (hi >= lo).all()
    assert ((hi >= 10) | (hi == 0)).all() and hi.max() <= 128
    b = np.clip(np.ceil((p - 0.5) / 0.1 - 1e-4).astype(int) - 1, 0, 14)
    tq = hi[b].astype(np.int32)
    _, _, st = idx.search(dev(qs), dev(p), k=10, ef=48, t=dev(tq), ef_max=128, stats=True)
    st = st.cpu().numpy()
    direct = (p == 1.0) | (p == 2.0)
    np.testing.assert_array_equal(st[~direct, 1], tq[~direct])
    assert (st[direct, 1] == 0).all() and (st[:, 5] == 0).all()
    idx.close()
