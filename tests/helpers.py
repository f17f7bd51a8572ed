"""Shared test helpers: cached workloads and graphs, and the top-k comparison
rule (ids identical except near-ties within 1e-5 relative; distances within
2e-5 relative of the FP64 oracle)."""
from __future__ import annotations

import functools

import numpy as np

import oracle
from paper_2605_02030_gb300 import inputs as I

TIE_RTOL = 1e-5
DIST_RTOL = 2e-5


@functools.lru_cache(maxsize=None)
def workload_arrays(name: str, n: int, nq: int, grid: float = 0.0, **kw):
    w = I.WORKLOADS[name].scaled(n=n, nq=nq, grid=grid, **kw)
    base = I.base_vectors(w)
    qs = I.query_vectors(w)
    p, k, ef = I.query_params(w)
    return w, base, qs, p, k, ef


@functools.lru_cache(maxsize=None)
def oracle_graphs(name: str, n: int, nq: int, grid: float = 0.0, **kw):
    w, base, *_ = workload_arrays(name, n, nq, grid, **kw)
    g1 = oracle.hnsw_build(base, 1, w.M, w.ef_construction, I.graph_levels(w, 1))
    g2 = oracle.hnsw_build(base, 2, w.M, w.ef_construction, I.graph_levels(w, 2))
    return g1, g2


def check_topk(base, q, p, got_ids, got_dist, ref_ids, k, what=""):
    """One query: got (ids, dist) against the oracle's ids ref_ids (ascending
    (S, id)).  Every returned id must carry its own L_p distance (FP64 oracle,
    2e-5 relative), the list must be ascending, and the id set may differ from
    the oracle's only by entries whose S ties the boundary within 1e-5."""
    p = float(np.float32(p))
    got_ids = np.asarray(got_ids[:k])
    got_dist = np.asarray(got_dist[:k], np.float64)
    ref_ids = np.asarray(ref_ids[:k])
    valid = got_ids >= 0
    assert valid.sum() == (ref_ids >= 0).sum(), f"{what}: result count {valid.sum()} vs {(ref_ids >= 0).sum()}"
    gi = got_ids[valid]
    assert len(set(gi.tolist())) == len(gi), f"{what}: duplicate ids"
    ref_S = {int(i): oracle.lp_sum(base[i], q, p) for i in set(gi.tolist()) | set(ref_ids[ref_ids >= 0].tolist())}
    for i, dd in zip(gi, got_dist[valid]):
        exp = ref_S[int(i)] ** (1.0 / p)
        assert abs(dd - exp) <= DIST_RTOL * max(exp, 1e-30), f"{what}: id {i} dist {dd} vs {exp}"
    assert np.all(np.diff(got_dist[valid]) >= -DIST_RTOL * np.abs(got_dist[valid][1:]) - 1e-30), f"{what}: not ascending"
    extra = set(gi.tolist()) - set(ref_ids.tolist())
    missing = set(ref_ids[ref_ids >= 0].tolist()) - set(gi.tolist())
    if extra or missing:
        kth = max(ref_S[int(i)] for i in ref_ids[ref_ids >= 0])
        for i in extra | missing:
            assert abs(ref_S[i] - kth) <= TIE_RTOL * max(kth, 1e-30), \
                f"{what}: id {i} S={ref_S[i]} differs from boundary {kth} beyond a near-tie"
    return len(extra)
