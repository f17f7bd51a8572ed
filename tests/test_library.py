"""Host-side checks of libuhnsw.so (no GPU): it builds, exports every entry
point of include/uhnsw.h, validates arguments before touching the device, and
its host graph builder matches the oracle's construction."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_2605_02030_gb300 import _build, inputs as I
from paper_2605_02030_gb300 import uhnsw as U

from helpers import workload_arrays

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    _build.build()
    return U.load_library()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "uhnsw.h")).read()
    declared = set(re.findall(r"\b(uhnsw_[a-z_]+)\s*\(", hdr))
    assert declared == set(U.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {_build.LIB}").read()
    for name in declared:
        assert re.search(rf"\bT {name}\b", out), f"{name} not exported"


def test_load_validation_errors(lib):
    base = np.zeros((4, 8), np.float32)
    h = C.c_void_p(0)
    assert lib.uhnsw_load(None, 4, 8, None, None, None, C.byref(h)) == -1
    assert b"base" in lib.uhnsw_last_error()
    g = {"num_levels": 1, "entry_point": 0, "max_degree0": 2, "max_degree": 2, "n": 4,
         "levels": [{"nodes": np.arange(4, dtype=np.int32), "offsets": np.array([0, 1, 2, 3, 4]),
                     "nbrs": np.array([1, 0, 3, 9], np.int32)}]}          # 9 is out of range
    s, keep = U._graph_struct(g)
    assert lib.uhnsw_load(base.ctypes.data, 4, 8, C.byref(s), None, None, C.byref(h)) == -1
    assert b"out of range" in lib.uhnsw_last_error()
    g["levels"][0]["nbrs"] = np.array([1, 0, 3, 2], np.int32)
    g["entry_point"] = 7
    s, keep = U._graph_struct(g)
    assert lib.uhnsw_load(base.ctypes.data, 4, 8, C.byref(s), None, None, C.byref(h)) == -1
    assert b"entry point" in lib.uhnsw_last_error()
    g["entry_point"] = 0
    g["max_degree0"] = 0
    s, keep = U._graph_struct(g)
    assert lib.uhnsw_load(base.ctypes.data, 4, 8, C.byref(s), None, None, C.byref(h)) == -1
    assert lib.uhnsw_load(base.ctypes.data, 4, 0, C.byref(s), None, None, C.byref(h)) == -1
    assert lib.uhnsw_load(base.ctypes.data, 4, 8, None, None, None, C.byref(h)) == -1
    # an upper level listing a node that is not on the level below
    g = {"num_levels": 2, "entry_point": 3, "max_degree0": 2, "max_degree": 2, "n": 4,
         "levels": [{"nodes": np.arange(4, dtype=np.int32), "offsets": np.array([0, 1, 2, 3, 4]),
                     "nbrs": np.array([1, 0, 3, 2], np.int32)},
                    {"nodes": np.array([3, 2], np.int32), "offsets": np.array([0, 0, 0]),
                     "nbrs": np.zeros(0, np.int32)}]}
    s, keep = U._graph_struct(g)
    assert lib.uhnsw_load(base.ctypes.data, 4, 8, C.byref(s), None, None, C.byref(h)) == -1
    assert b"ascending" in lib.uhnsw_last_error()


def test_search_validation_errors(lib):
    assert lib.uhnsw_search(None, None, None, None, None, 1, 10, 64, None, None, None, None) == -1
    assert lib.uhnsw_verify(None, None, None, None, 1, 1, 1, None, None, None, None) == -1
    assert lib.uhnsw_exact(None, None, None, 1, 1, None, None, None) == -1
    assert lib.uhnsw_index_info(None, None, None, None, None, None) == -1


def test_build_graph_validation(lib):
    base = np.zeros((10, 4), np.float32)
    lv = np.zeros(10, np.int32)
    h = C.c_void_p(0)
    assert lib.uhnsw_build_graph(base.ctypes.data, 10, 4, 5, 4, 10, lv.ctypes.data, 1, C.byref(h)) == -1
    assert lib.uhnsw_build_graph(base.ctypes.data, 10, 4, 0, 4, 10, lv.ctypes.data, 1, C.byref(h)) == -1
    assert lib.uhnsw_build_graph(base.ctypes.data, 10, 4, 1, 1, 10, lv.ctypes.data, 1, C.byref(h)) == -1
    lv[3] = -2
    assert lib.uhnsw_build_graph(base.ctypes.data, 10, 4, 1, 4, 10, lv.ctypes.data, 1, C.byref(h)) == -1


def _same_graph(a, b):
    if a["num_levels"] != b["num_levels"] or a["entry_point"] != b["entry_point"]:
        return False
    for x, y in zip(a["levels"], b["levels"]):
        for key in ("nodes", "offsets", "nbrs"):
            if not np.array_equal(x[key], y[key]):
                return False
    return True


@pytest.mark.parametrize("case", [("sift1m", 3000, 0.0, dict(M=8, ef_construction=40)),
                                  ("mixture10k", 3000, 1 / 16, dict(M=8, ef_construction=30))])
def test_builder_single_thread_equals_oracle(lib, case):
    """Integer data (and data on a 1/16 grid) make FP32 L1/L2 sums exact, so
    one-thread insertion reproduces the oracle's FP64 construction exactly."""
    name, n, grid, kw = case
    w, base, *_ = workload_arrays(name, n, 4, grid, **kw)
    for metric in (1, 2):
        lv = I.graph_levels(w, metric)
        go = oracle.hnsw_build(base, metric, w.M, w.ef_construction, lv)
        gp = U.build_graph(base, metric, w.M, w.ef_construction, lv, threads=1)
        assert _same_graph(go, gp), (name, metric)


def test_builder_l05_single_thread_equals_oracle(lib):
    """The L0.5 graph of U-HNSW-E (metric 3) on 0/1 data, where every |d_j|^(1/2)
    is 0 or 1 and the FP32 sums are exact: one-thread insertion reproduces the
    oracle's FP64 construction exactly."""
    r = np.random.default_rng(13)
    base = r.integers(0, 2, size=(1500, 32)).astype(np.float32)
    lv = I.hnsw_levels(len(base), 8, 5)
    go = oracle.hnsw_build(base, 3, 8, 30, lv)
    gp = U.build_graph(base, 3, 8, 30, lv, threads=1)
    assert _same_graph(go, gp)


def test_builder_lp_single_thread_equals_oracle(lib):
    """A graph under a general L_p (p = 0.8, metric 5) on 0/1 data, where every
    |d_j|^0.8 is exactly 0 or 1: one-thread insertion reproduces the oracle's
    FP64 construction under the same p exactly; p = 1 through the same entry
    point is the L1 graph, and p = 1.5 the L1.5 graph (metric 4)."""
    r = np.random.default_rng(31)
    base = r.integers(0, 2, size=(1500, 32)).astype(np.float32)
    lv = I.hnsw_levels(len(base), 8, 5)
    go = oracle.hnsw_build(base, None, 8, 30, lv, base_p=0.8)
    gp = U.build_graph(base, U.BASE_LP, 8, 30, lv, threads=1, p=0.8)
    assert _same_graph(go, gp)
    g1 = U.build_graph(base, U.BASE_LP, 8, 30, lv, threads=1, p=1.0)
    assert _same_graph(oracle.hnsw_build(base, 1, 8, 30, lv), g1)
    g15 = U.build_graph(base, U.BASE_LP, 8, 30, lv, threads=1, p=1.5)
    assert _same_graph(oracle.hnsw_build(base, 4, 8, 30, lv), g15)
    assert _same_graph(U.build_graph(base, U.BASE_L15, 8, 30, lv, threads=1), g15)


def test_lp_validation(lib):
    """Base p outside (0, 2], an unknown metric code, or a first slot whose p
    is not below the second's are refused before any device work."""
    base = np.zeros((10, 4), np.float32)
    lv = np.zeros(10, np.int32)
    h = C.c_void_p(0)
    for p in (0.0, -0.5, 2.5, float("nan")):
        assert lib.uhnsw_build_graph_lp(base.ctypes.data, 10, 4, p, 4, 10, lv.ctypes.data, 1, 0,
                                        C.byref(h)) == -1
        assert b"outside" in lib.uhnsw_last_error()
    g = {"num_levels": 1, "entry_point": 0, "max_degree0": 2, "max_degree": 2, "n": 4,
         "levels": [{"nodes": np.arange(4, dtype=np.int32), "offsets": np.array([0, 1, 2, 3, 4]),
                     "nbrs": np.array([1, 0, 3, 2], np.int32)}]}
    s, keep = U._graph_struct(g)
    b4 = np.zeros((4, 8), np.float32)
    for metrics, bp, what in (((5, 2), (0.0, 0.0), b"outside"), ((5, 2), (2.5, 0.0), b"outside"),
                              ((5, 5), (0.8, 0.8), b"below"), ((5, 1), (1.2, 0.0), b"below"),
                              ((6, 2), (0.0, 0.0), b"uhnsw_base_metric")):
        o = U._LoadOpts()
        o.base_metric[0], o.base_metric[1] = metrics
        o.base_p[0], o.base_p[1] = bp
        assert lib.uhnsw_load(b4.ctypes.data, 4, 8, C.byref(s), C.byref(s), C.byref(o),
                              C.byref(h)) == -1
        assert what in lib.uhnsw_last_error(), (metrics, bp)


def test_builder_parallel_invariants(lib):
    w, base, *_ = workload_arrays("sift1m", 8000, 4, 0.0, M=12, ef_construction=60)
    lv = I.graph_levels(w, 2)
    g = U.build_graph(base, 2, w.M, w.ef_construction, lv, threads=4)
    assert g["num_levels"] == lv.max() + 1 and lv[g["entry_point"]] == lv.max()
    for l, L in enumerate(g["levels"]):
        np.testing.assert_array_equal(L["nodes"], np.nonzero(lv >= l)[0])
        deg = np.diff(L["offsets"])
        assert deg.max() <= (2 * w.M if l == 0 else w.M)
        assert (lv[L["nbrs"]] >= l).all()
    # Pruned reverse links leave a few nodes without an in-link on layer 0 in
    # any HNSW build (the oracle's too), so reachability from the entry point
    # is compared with the single-threaded build rather than required to be 1.
    def reach(gr):
        L0 = gr["levels"][0]
        seen = np.zeros(w.n, bool)
        seen[gr["entry_point"]] = True
        fr = [gr["entry_point"]]
        while fr:
            nxt = []
            for v in fr:
                for u in L0["nbrs"][L0["offsets"][v]:L0["offsets"][v + 1]]:
                    if not seen[u]:
                        seen[u] = True
                        nxt.append(int(u))
            fr = nxt
        return seen.mean()

    g1 = U.build_graph(base, 2, w.M, w.ef_construction, lv, threads=1)
    assert reach(g) >= reach(g1) - 0.01


def test_plan_t_picks_the_smallest_t_per_p_bin(lib):
    """uhnsw_plan_t on hand-made idealized-recall counts (K = 4, t_max = 6):
    the smallest t whose mean count over a bin's queries reaches target * K."""
    counts = np.array([[1, 2, 3, 4, 4, 4],     # p = 0.55 -> bin 0
                       [0, 1, 2, 2, 3, 4],     # p = 0.58 -> bin 0
                       [2, 4, 4, 4, 4, 4],     # p = 0.75 -> bin 2
                       [0, 0, 0, 1, 1, 2]],    # p = 1.95 -> bin 14
                      np.int32)
    p = np.array([0.55, 0.58, 0.75, 1.95], np.float32)
    # bin 0 means: 0.5, 1.5, 2.5, 3, 3.5, 4 (out of 4)
    np.testing.assert_array_equal(U.plan_t(counts, p, 4, 0.75)[[0, 1, 2, 14]], [4, 0, 2, 6])
    np.testing.assert_array_equal(U.plan_t(counts, p, 4, 0.875)[[0, 2]], [5, 2])
    np.testing.assert_array_equal(U.plan_t(counts, p, 4, 1.0)[[0, 2, 14]], [6, 2, 6])
    # p at a bin's upper edge belongs to that bin; below p_lo goes to bin 0
    out = U.plan_t(counts[:1], np.array([0.6], np.float32), 4, 1.0)
    assert out[0] == 4 and out[1] == 0
    out = U.plan_t(counts[:1], np.array([0.1], np.float32), 4, 1.0)
    assert out[0] == 4
    with pytest.raises(U.UHNSWError):
        U.plan_t(counts, p, 4, 1.5)
    with pytest.raises(U.UHNSWError):
        U.plan_t(counts, p, 7, 0.5)          # K above t_max
