"""U-HNSW oracle: TEST INFRASTRUCTURE ONLY.

Python bindings (ctypes) for ``uhnsw_oracle.c``, the plain single-threaded
FP64 CPU restatement of the U-HNSW query path (arxiv 2605.02030, Section 3.1,
Algorithm 1) and of the HNSW routines it relies on (Section 2.2).  Only the
tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may use
this package; the library under ``paper_2605_02030_gb300`` never imports it.

Pinned by ``tests/test_oracle.py`` (closed forms, library routines, hand-
derived graphs, invariants).  ``hnsw_build`` is pinned by hand-derived small
graphs and, at efConstruction >= N, by a brute-force insertion (every
reachable earlier node ranked); at smaller efConstruction its graph follows
the insertion beam, whose search is pinned on its own, and the index quality
is checked (connectivity, degree bounds, search recall).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "uhnsw_oracle.c")
_SRC_THREADS = os.path.join(_HERE, "batch_threads.c")
_LIB = os.path.join(_HERE, "_uhnsw_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no SIMD flags, no fast-math)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_THREADS))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC,
               _SRC_THREADS, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _CSR(C.Structure):
    _fields_ = [
        ("num_levels", C.c_int32),
        ("entry_point", C.c_int32),
        ("max_degree0", C.c_int32),
        ("max_degree", C.c_int32),
        ("n", C.c_int64),
        ("count", C.POINTER(C.c_int32)),
        ("nodes", C.POINTER(C.c_void_p)),
        ("offsets", C.POINTER(C.c_void_p)),
        ("nbrs", C.POINTER(C.c_void_p)),
    ]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.c_void_p
    lib.oracle_lp_sum.restype = C.c_double
    lib.oracle_lp_sum.argtypes = [P, P, C.c_int32, C.c_double]
    lib.oracle_base_dist.restype = C.c_double
    lib.oracle_base_dist.argtypes = [P, P, C.c_int32, C.c_int32]
    lib.oracle_exact_knn.restype = C.c_int
    lib.oracle_exact_knn.argtypes = [P, C.c_int64, C.c_int32, P, C.c_int64, P, C.c_int32, P, P]
    lib.oracle_select_heuristic.restype = C.c_int32
    lib.oracle_select_heuristic.argtypes = [P, C.c_int32, C.c_int32, P, P, C.c_int32, C.c_int32, P]
    lib.oracle_hnsw_build.restype = P
    lib.oracle_hnsw_build.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                      C.c_int32, P, P]
    lib.oracle_hnsw_build_p.restype = P
    lib.oracle_hnsw_build_p.argtypes = [P, C.c_int64, C.c_int32, C.c_double, C.c_int32, C.c_int32,
                                        C.c_int32, P, P]
    lib.oracle_graph_free.argtypes = [P]
    lib.oracle_graph_num_levels.restype = C.c_int32
    lib.oracle_graph_num_levels.argtypes = [P]
    lib.oracle_graph_entry.restype = C.c_int32
    lib.oracle_graph_entry.argtypes = [P]
    lib.oracle_graph_level_size.argtypes = [P, C.c_int32, P, P]
    lib.oracle_graph_level_copy.argtypes = [P, C.c_int32, P, P, P]
    lib.oracle_hnsw_search.restype = C.c_int
    lib.oracle_hnsw_search.argtypes = [C.POINTER(_CSR), P, C.c_int32, C.c_int32, P, C.c_int32,
                                       C.c_int32, P, P, P]
    lib.oracle_hnsw_search_p.restype = C.c_int
    lib.oracle_hnsw_search_p.argtypes = [C.POINTER(_CSR), P, C.c_int32, C.c_double, P, C.c_int32,
                                         C.c_int32, P, P, P]
    lib.oracle_hnsw_search_w.restype = C.c_int
    lib.oracle_hnsw_search_w.argtypes = [C.POINTER(_CSR), P, C.c_int32, C.c_double, P, C.c_int32,
                                         C.c_int32, C.c_int32, P, P, P]
    lib.oracle_verify_exact.restype = C.c_int
    lib.oracle_verify_exact.argtypes = [P, C.c_int32, P, C.c_double, P, C.c_int32, C.c_int32,
                                        C.c_int32, P, P, P]
    lib.oracle_verify_paper.restype = C.c_int
    lib.oracle_verify_paper.argtypes = [P, C.c_int32, P, C.c_double, P, C.c_int32, C.c_int32,
                                        C.c_int32, C.c_float, P, P, P, P]
    lib.oracle_uhnsw_query.restype = C.c_int
    lib.oracle_uhnsw_query.argtypes = [C.POINTER(_CSR), C.POINTER(_CSR), C.c_int32, C.c_int32, P,
                                       C.c_int32, P, C.c_float, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_float, C.c_int32, C.c_float, C.c_int32, P, P, P]
    lib.oracle_uhnsw_batch_threads.restype = C.c_int
    lib.oracle_uhnsw_batch_threads.argtypes = [C.POINTER(_CSR), C.POINTER(_CSR), C.c_int32,
                                               C.c_int32, P, C.c_int32, P, P, C.c_int64,
                                               C.c_int32, C.c_int32, C.c_int32, C.c_float,
                                               C.c_int32, C.c_float, C.c_int32, C.c_int32, P, P]
    lib.oracle_uhnsw_query_w.restype = C.c_int
    lib.oracle_uhnsw_query_w.argtypes = [C.POINTER(_CSR), C.POINTER(_CSR), C.c_double, C.c_double,
                                         P, C.c_int32, P, C.c_float, C.c_int32, C.c_int32,
                                         C.c_int32, C.c_float, C.c_int32, C.c_float, C.c_int32,
                                         C.c_int32, P, P, P]
    lib.oracle_uhnsw_query_trav.restype = C.c_int
    lib.oracle_uhnsw_query_trav.argtypes = [C.POINTER(_CSR), C.POINTER(_CSR), C.c_double,
                                            C.c_double, P, P, C.c_int32, P, C.c_float, C.c_int32,
                                            C.c_int32, C.c_int32, C.c_float, C.c_int32, C.c_float,
                                            C.c_int32, C.c_int32, C.c_double, P, P, P, P]
    lib.oracle_uhnsw_query_p.restype = C.c_int
    lib.oracle_uhnsw_query_p.argtypes = [C.POINTER(_CSR), C.POINTER(_CSR), C.c_double, C.c_double,
                                         P, C.c_int32, P, C.c_float, C.c_int32, C.c_int32,
                                         C.c_int32, C.c_float, C.c_int32, C.c_float, C.c_int32, P,
                                         P, P]
    _lib = lib
    return lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- distances
def lp_sum(x, q, p: float) -> float:
    """S = sum_j |x_j - q_j|^p in FP64 (Section 2.1)."""
    x, q = _f32(x), _f32(q)
    return _load().oracle_lp_sum(_ptr(x), _ptr(q), x.shape[-1], float(p))


# Base metrics of the graphs (metric codes): 1 = L1, sum |d_j|; 2 = squared
# L2, sum d_j^2; 3 = L0.5 without its root, sum |d_j|^(1/2); 4 = L1.5 without
# its root, sum |d_j|^(3/2).  METRIC_P is the p of each.  U-HNSW uses G1 (L1) and G2 (L2) with cutoff 1.4; U-HNSW-E
# (Section 4.5) uses G0.5 (L0.5) and G1 (L1) with cutoff 0.6.
METRIC_P = {1: 1.0, 2: 2.0, 3: 0.5, 4: 1.5}


def _bp(p) -> float:
    """A graph's base p as the FP32 value it is stored as, widened to FP64:
    a graph built under L_bp uses S_bp = sum |d_j|^bp (the fixed-p HNSW of
    Section 4.3, one graph per p)."""
    bp = float(np.float32(p))
    if not 0.0 < bp <= 2.0:
        raise ValueError(f"base p {p} outside (0, 2]")
    return bp


def base_dist(x, q, metric: int) -> float:
    """metric 1: sum |d_j| (L1); 2: sum d_j^2 (squared L2); 3: sum |d_j|^(1/2)
    (L0.5); 4: sum |d_j|^(3/2) (L1.5)."""
    x, q = _f32(x), _f32(q)
    return _load().oracle_base_dist(_ptr(x), _ptr(q), x.shape[-1], int(metric))


# ---------------------------------------------------------------- O1
def exact_knn(base, queries, p, k: int):
    """Exact top-k under each query's L_p: (ids int64 [nq,k], S float64 [nq,k]),
    ascending by (S, id); padded with -1 / inf when n < k."""
    base, queries = _f32(base), _f32(queries)
    p = _f32(np.broadcast_to(np.asarray(p, np.float32), (queries.shape[0],)))
    nq = queries.shape[0]
    ids = np.empty((nq, k), np.int64)
    S = np.empty((nq, k), np.float64)
    rc = _load().oracle_exact_knn(_ptr(base), base.shape[0], base.shape[1], _ptr(queries), nq,
                                  _ptr(p), k, _ptr(ids), _ptr(S))
    if rc != 0:
        raise ValueError(f"oracle_exact_knn: {rc}")
    return ids, S


# ---------------------------------------------------------------- O2
def select_heuristic(base, cand, cand_d, m: int, metric: int):
    """HNSW neighbour-selection heuristic over `cand` (sorted by cand_d)."""
    base = _f32(base)
    cand = np.ascontiguousarray(cand, np.int64)
    cand_d = np.ascontiguousarray(cand_d, np.float64)
    out = np.empty(max(m, 1), np.int32)
    r = _load().oracle_select_heuristic(_ptr(base), base.shape[1], metric, _ptr(cand), _ptr(cand_d),
                                        len(cand), m, _ptr(out))
    return out[:r].copy()


def hnsw_build(base, metric: int | None, M: int, ef_construction: int, levels,
               M0: int | None = None, base_p: float | None = None):
    """HNSW graph under L1 (metric=1), L2 (2), L0.5 (3) or L1.5 (4), or, with
    metric None and base_p given, under L_base_p, as a CSR dict:
    {num_levels, entry_point, max_degree0, max_degree, n,
     levels: [{nodes int32, offsets int64, nbrs int32}, ...]} (level 0 nodes = all ids)."""
    base = _f32(base)
    levels = np.ascontiguousarray(levels, np.int32)
    n, d = base.shape
    M0 = 2 * M if M0 is None else M0
    lib = _load()
    st = C.c_int32(0)
    if metric is None:
        g = lib.oracle_hnsw_build_p(_ptr(base), n, d, _bp(base_p), M, M0, ef_construction,
                                    _ptr(levels), C.byref(st))
    else:
        g = lib.oracle_hnsw_build(_ptr(base), n, d, metric, M, M0, ef_construction, _ptr(levels),
                                  C.byref(st))
    if not g:
        raise ValueError(f"oracle_hnsw_build: status {st.value}")
    try:
        L = lib.oracle_graph_num_levels(g)
        out = {"num_levels": L, "entry_point": lib.oracle_graph_entry(g), "max_degree0": M0,
               "max_degree": M, "n": n, "levels": []}
        for l in range(L):
            nn, ne = C.c_int64(0), C.c_int64(0)
            lib.oracle_graph_level_size(g, l, C.byref(nn), C.byref(ne))
            nodes = np.empty(nn.value, np.int32)
            offs = np.empty(nn.value + 1, np.int64)
            nbrs = np.empty(max(ne.value, 1), np.int32)
            lib.oracle_graph_level_copy(g, l, _ptr(nodes), _ptr(offs), _ptr(nbrs))
            out["levels"].append({"nodes": nodes, "offsets": offs, "nbrs": nbrs[:ne.value].copy()})
    finally:
        lib.oracle_graph_free(g)
    return out


class _CSRHolder:
    """Keeps the numpy arrays behind a ctypes CSR struct alive."""

    def __init__(self, g):
        L = g["num_levels"]
        self.arrays = []
        cnt = np.array([len(lv["nodes"]) for lv in g["levels"]], np.int32)
        nodes = (C.c_void_p * L)()
        offs = (C.c_void_p * L)()
        nbrs = (C.c_void_p * L)()
        for l, lv in enumerate(g["levels"]):
            a = np.ascontiguousarray(lv["nodes"], np.int32)
            b = np.ascontiguousarray(lv["offsets"], np.int64)
            c = np.ascontiguousarray(lv["nbrs"], np.int32)
            if c.size == 0:
                c = np.zeros(1, np.int32)
            self.arrays += [a, b, c]
            nodes[l] = a.ctypes.data
            offs[l] = b.ctypes.data
            nbrs[l] = c.ctypes.data
        self.arrays += [cnt, nodes, offs, nbrs]
        self.s = _CSR(L, g["entry_point"], g["max_degree0"], g["max_degree"], g["n"],
                      cnt.ctypes.data_as(C.POINTER(C.c_int32)),
                      C.cast(nodes, C.POINTER(C.c_void_p)), C.cast(offs, C.POINTER(C.c_void_p)),
                      C.cast(nbrs, C.POINTER(C.c_void_p)))


# ---------------------------------------------------------------- O3
def hnsw_search(graph, base, q, metric: int | None, ef: int, t: int, base_p: float | None = None,
                width: int | None = None):
    """KnnSearch(q, t) with beam ef on a CSR graph (base metric by code, or
    L_base_p when metric is None): (ids int64 [t], base dist float64 [t],
    number of base-distance evaluations).  With `width` given, the layer-0
    beam expands that many entries per step (the GPU's fast mode; width = 1
    is HNSW's order through a second, independent routine)."""
    base, q = _f32(base), _f32(q)
    h = _CSRHolder(graph)
    ids = np.empty(t, np.int64)
    dd = np.empty(t, np.float64)
    nd = C.c_int64(0)
    if width is not None:
        bp = _bp(base_p) if metric is None else METRIC_P[int(metric)]
        rc = _load().oracle_hnsw_search_w(C.byref(h.s), _ptr(base), base.shape[1], bp, _ptr(q),
                                          ef, t, int(width), _ptr(ids), _ptr(dd), C.byref(nd))
    elif metric is None:
        rc = _load().oracle_hnsw_search_p(C.byref(h.s), _ptr(base), base.shape[1], _bp(base_p),
                                          _ptr(q), ef, t, _ptr(ids), _ptr(dd), C.byref(nd))
    else:
        rc = _load().oracle_hnsw_search(C.byref(h.s), _ptr(base), base.shape[1], metric, _ptr(q),
                                        ef, t, _ptr(ids), _ptr(dd), C.byref(nd))
    if rc != 0:
        raise ValueError(f"oracle_hnsw_search: {rc}")
    return ids, dd, nd.value


# ---------------------------------------------------------------- O4
def verify_exact(base, q, p: float, cand, k: int, abandon: bool = True):
    """Top-k by (S, id) over the candidate ids (-1 = absent): (ids, S, terms)."""
    base, q = _f32(base), _f32(q)
    cand = np.ascontiguousarray(cand, np.int32)
    ids = np.empty(k, np.int64)
    S = np.empty(k, np.float64)
    nt = C.c_int64(0)
    rc = _load().oracle_verify_exact(_ptr(base), base.shape[1], _ptr(q), float(np.float32(p)),
                                     _ptr(cand), len(cand), k, int(abandon), _ptr(ids), _ptr(S),
                                     C.byref(nt))
    if rc != 0:
        raise ValueError(f"oracle_verify_exact: {rc}")
    return ids, S, nt.value


def verify_paper(base, q, p: float, cand, k: int, kappa: int, tau: float):
    """Algorithm 1 lines 6-10: (ids, S, n_lp, n_batches)."""
    base, q = _f32(base), _f32(q)
    cand = np.ascontiguousarray(cand, np.int32)
    ids = np.empty(k, np.int64)
    S = np.empty(k, np.float64)
    nl, nb = C.c_int64(0), C.c_int64(0)
    rc = _load().oracle_verify_paper(_ptr(base), base.shape[1], _ptr(q), float(np.float32(p)),
                                     _ptr(cand), len(cand), k, kappa, float(tau), _ptr(ids),
                                     _ptr(S), C.byref(nl), C.byref(nb))
    if rc != 0:
        raise ValueError(f"oracle_verify_paper: {rc}")
    return ids, S, nl.value, nb.value


# ---------------------------------------------------------------- Algorithm 1
def uhnsw_query(g1, g2, base, q, p: float, k: int, ef: int, t: int = 0, tau: float = 0.92,
                kappa: int = 0, cutoff: float = 1.4, mode: int = 0, metrics=(1, 2), _holders=None,
                base_p=None, width: int = 1):
    """One query of Algorithm 1: (ids int64 [k], dist float64 [k], stats [N_b, N_p, terms]).
    g1 / g2 are the graphs routed for p <= cutoff / p > cutoff, under the base
    metrics `metrics` (U-HNSW: (1, 2); U-HNSW-E: (3, 1) with cutoff 0.6), or,
    when base_p = (pa, pb) is given, under L_pa and L_pb (a fixed HNSW at p:
    the same L_p graph in both slots, base_p = (p, p)).  width > 1 runs
    the layer-0 beam in the GPU's fast mode (that many expansions per step)."""
    base, q = _f32(base), _f32(q)
    h1 = _holders[0] if _holders else _CSRHolder(g1)
    h2 = _holders[1] if _holders else _CSRHolder(g2)
    ids = np.empty(k, np.int64)
    dist = np.empty(k, np.float64)
    st = np.zeros(3, np.int64)
    if width != 1:
        bpa, bpb = ((_bp(base_p[0]), _bp(base_p[1])) if base_p is not None
                    else (METRIC_P[int(metrics[0])], METRIC_P[int(metrics[1])]))
        rc = _load().oracle_uhnsw_query_w(C.byref(h1.s), C.byref(h2.s), bpa, bpb, _ptr(base),
                                          base.shape[1], _ptr(q), float(p), k, ef, t, float(tau),
                                          kappa, float(cutoff), mode, int(width), _ptr(ids),
                                          _ptr(dist), _ptr(st))
    elif base_p is not None:
        rc = _load().oracle_uhnsw_query_p(C.byref(h1.s), C.byref(h2.s), _bp(base_p[0]),
                                          _bp(base_p[1]), _ptr(base), base.shape[1], _ptr(q),
                                          float(p), k, ef, t, float(tau), kappa, float(cutoff),
                                          mode, _ptr(ids), _ptr(dist), _ptr(st))
    else:
        rc = _load().oracle_uhnsw_query(C.byref(h1.s), C.byref(h2.s), int(metrics[0]),
                                        int(metrics[1]), _ptr(base), base.shape[1], _ptr(q),
                                        float(p), k, ef, t, float(tau), kappa, float(cutoff), mode,
                                        _ptr(ids), _ptr(dist), _ptr(st))
    if rc != 0:
        raise ValueError(f"oracle_uhnsw_query: {rc}")
    return ids, dist, st


def uhnsw_query_trav(g1, g2, base, trav, q, p: float, k: int, ef: int, t: int = 0,
                     tau: float = 0.92, kappa: int = 0, cutoff: float = 1.4, mode: int = 0,
                     metrics=(1, 2), width: int = 1, tie_tol: float = 0.0, _holders=None):
    """One query of Algorithm 1 in the precision form: the graph search
    computes base distances (FP64) on `trav`, rows of the same shape as
    `base` (the FP16 / BF16 copy's values as FP32), verification and the
    returned distances use `base`.  A direct query (p = 1 or 2) ranks its
    whole beam by the exact base distance on `base`.  Returns (ids [k], dist
    [k], C [t' or ef'] (the candidate list, -1 padded), stats [N_b, N_p,
    terms, near-tie comparisons of the search at relative tolerance
    tie_tol])."""
    base, trav, q = _f32(base), _f32(trav), _f32(q)
    if trav.shape != base.shape:
        raise ValueError("trav must have the shape of base")
    h1 = _holders[0] if _holders else _CSRHolder(g1)
    h2 = _holders[1] if _holders else _CSRHolder(g2)
    bpa, bpb = METRIC_P[int(metrics[0])], METRIC_P[int(metrics[1])]
    tt = max(t if t > 0 else ef, k)
    cap = max(ef, tt)
    ids = np.empty(k, np.int64)
    dist = np.empty(k, np.float64)
    cand = np.full(cap, -1, np.int64)
    st = np.zeros(4, np.int64)
    rc = _load().oracle_uhnsw_query_trav(C.byref(h1.s), C.byref(h2.s), bpa, bpb, _ptr(base),
                                         _ptr(trav), base.shape[1], _ptr(q), float(p), k, ef, t,
                                         float(tau), kappa, float(cutoff), mode, int(width),
                                         float(tie_tol), _ptr(ids), _ptr(dist), _ptr(cand),
                                         _ptr(st))
    if rc != 0:
        raise ValueError(f"oracle_uhnsw_query_trav: {rc}")
    return ids, dist, cand, st


def uhnsw_batch(g1, g2, base, queries, p, k, ef, t=0, tau=0.92, kappa=0, cutoff=1.4, mode=0,
                metrics=(1, 2), base_p=None, width=1):
    """Algorithm 1 over a batch (per-query p, k, ef arrays or scalars).
    Returns ids int64 [nq, kmax] and dist float64 [nq, kmax] (-1 / inf padded)."""
    queries = _f32(queries)
    nq = queries.shape[0]
    p = np.broadcast_to(np.asarray(p, np.float32), (nq,))
    k = np.broadcast_to(np.asarray(k, np.int32), (nq,))
    ef = np.broadcast_to(np.asarray(ef, np.int32), (nq,))
    kmax = int(k.max())
    holders = (_CSRHolder(g1), _CSRHolder(g2))
    ids = np.full((nq, kmax), -1, np.int64)
    dist = np.full((nq, kmax), np.inf, np.float64)
    stats = np.zeros((nq, 3), np.int64)
    for i in range(nq):
        a, b, s = uhnsw_query(g1, g2, base, queries[i], float(p[i]), int(k[i]), int(ef[i]), t, tau,
                              kappa, cutoff, mode, metrics, _holders=holders, base_p=base_p,
                              width=width)
        ids[i, :k[i]] = a
        dist[i, :k[i]] = b
        stats[i] = s
    return ids, dist, stats


def uhnsw_batch_threads(g1, g2, base, queries, p, k: int, ef: int, threads: int, t=0, tau=0.92,
                        kappa=0, cutoff=1.4, mode=0, metrics=(1, 2), _holders=None):
    """Algorithm 1 over a batch with one k and ef, the queries spread over
    `threads` host threads (each query one single-threaded oracle call).
    Returns ids int64 [nq, k] and dist float64 [nq, k]."""
    base = _f32(base)
    queries = _f32(queries)
    nq = queries.shape[0]
    p = _f32(np.broadcast_to(np.asarray(p, np.float32), (nq,)))
    h1, h2 = _holders if _holders else (_CSRHolder(g1), _CSRHolder(g2))
    ids = np.empty((nq, k), np.int64)
    dist = np.empty((nq, k), np.float64)
    rc = _load().oracle_uhnsw_batch_threads(C.byref(h1.s), C.byref(h2.s), int(metrics[0]),
                                            int(metrics[1]), _ptr(base), base.shape[1],
                                            _ptr(queries), _ptr(p), nq, k, ef, t, float(tau),
                                            kappa, float(cutoff), mode, int(threads), _ptr(ids),
                                            _ptr(dist))
    if rc != 0:
        raise ValueError(f"oracle_uhnsw_batch_threads: {rc}")
    return ids, dist


def recall(found_ids, true_ids, k=None) -> float:
    """Mean over queries of |S* n S| / K (Section 4.1.2)."""
    found_ids = np.asarray(found_ids)
    true_ids = np.asarray(true_ids)
    nq = found_ids.shape[0]
    tot = 0.0
    for i in range(nq):
        kk = true_ids.shape[1] if k is None else int(np.broadcast_to(k, (nq,))[i])
        tru = set(int(v) for v in true_ids[i, :kk] if v >= 0)
        got = set(int(v) for v in found_ids[i, :kk] if v >= 0)
        tot += len(tru & got) / kk
    return tot / max(nq, 1)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
