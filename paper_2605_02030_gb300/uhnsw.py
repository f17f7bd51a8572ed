"""Python binding of the C ABI in include/uhnsw.h (argument marshalling only).

Every step of the query path runs in libuhnsw.so's CUDA kernels; this module
passes pointers and sizes.  torch provides device memory and streams.  The
library must have been built (``paper_2605_02030_gb300.build()``); a missing
library raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

MAX_LEVELS = 16
MAX_EF = 512
NSTATS = 8
STAT_NAMES = ("nb", "np", "terms", "expansions", "resets", "status", "graph", "adj")
DTYPES = {"f32": 0, "f16": 1, "bf16": 2}
MODES = {"exact": 0, "paper": 1}

_lib = None


class UHNSWError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"uhnsw error {code}: {msg}")
        self.code = code


class _Graph(C.Structure):
    _fields_ = [
        ("num_levels", C.c_int32),
        ("entry_point", C.c_int32),
        ("max_degree0", C.c_int32),
        ("max_degree", C.c_int32),
        ("level_count", C.c_void_p),
        ("level_nodes", C.c_void_p * MAX_LEVELS),
        ("level_offsets", C.c_void_p * MAX_LEVELS),
        ("level_nbrs", C.c_void_p * MAX_LEVELS),
    ]


class _LoadOpts(C.Structure):
    _fields_ = [("traverse_dtype", C.c_int32), ("base_metric", C.c_int32 * 2),
                ("base_p", C.c_float * 2), ("reserved", C.c_int32 * 3)]


# Base metrics (uhnsw_base_metric): 1 = L1, 2 = squared L2, 3 = L0.5 sum,
# 4 = L1.5 sum, 5 = the L_p sum of a slot's base_p (any 0 < p <= 2).
BASE_L1, BASE_L2, BASE_L05, BASE_L15, BASE_LP = 1, 2, 3, 4, 5
U_HNSW = (BASE_L1, BASE_L2)        # G1 and G2, cutoff 1.4
U_HNSW_E = (BASE_L05, BASE_L1)     # G0.5 and G1, cutoff 0.6 (Section 4.5)


class _SearchOpts(C.Structure):
    _fields_ = [
        ("t", C.c_int32),
        ("kappa", C.c_int32),
        ("tau", C.c_float),
        ("cutoff", C.c_float),
        ("verify_mode", C.c_int32),
        ("search_width", C.c_int32),
        ("persistent", C.c_int32),
        ("use_graph", C.c_int32),
        ("ef_max", C.c_int32),
        ("query_threads", C.c_int32),
        ("stats", C.c_void_p),
        ("stage_bytes", C.c_int32),
        ("team_lanes", C.c_int32),
        ("kernel_events", C.c_void_p),
        ("t_per_query", C.c_void_p),
        ("tau_per_query", C.c_void_p),
        ("hash_bits", C.c_int32),
        ("verify_groups", C.c_int32),
    ]


EXPORTS = ("uhnsw_load", "uhnsw_search", "uhnsw_search_host", "uhnsw_search_host_async", "uhnsw_verify", "uhnsw_exact",
           "uhnsw_idealized_recall", "uhnsw_plan_t",
           "uhnsw_exact_static", "uhnsw_server_create", "uhnsw_server_submit", "uhnsw_server_poll",
           "uhnsw_server_wait", "uhnsw_server_replay", "uhnsw_server_stats",
           "uhnsw_server_destroy", "uhnsw_autotune", "uhnsw_autotune_save", "uhnsw_autotune_load",
           "uhnsw_index_info", "uhnsw_device_status", "uhnsw_free", "uhnsw_last_error",
           "uhnsw_build_graph", "uhnsw_build_graph_gpu", "uhnsw_build_graph_lp",
           "uhnsw_built_graph", "uhnsw_built_free", "uhnsw_probe_sfu", "uhnsw_probe_gather")


def library_path() -> str:
    return _build.LIB


def load_library():
    """Loads libuhnsw.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run paper_2605_02030_gb300.build() first")
    lib = C.CDLL(path)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    lib.uhnsw_last_error.restype = C.c_char_p
    lib.uhnsw_last_error.argtypes = []
    lib.uhnsw_load.restype = C.c_int
    lib.uhnsw_load.argtypes = [P, I64, I32, P, P, P, P]
    lib.uhnsw_search.restype = C.c_int
    lib.uhnsw_search.argtypes = [P, P, P, P, P, I64, I32, I32, P, P, P, P]
    lib.uhnsw_search_host.restype = C.c_int
    lib.uhnsw_search_host.argtypes = [P, P, P, P, P, I64, I32, I32, P, P, P, P]
    lib.uhnsw_search_host_async.restype = C.c_int
    lib.uhnsw_search_host_async.argtypes = [P, P, P, P, P, I64, I32, I32, P, P, P, P]
    lib.uhnsw_verify.restype = C.c_int
    lib.uhnsw_verify.argtypes = [P, P, P, P, I32, I32, I64, P, P, P, P]
    lib.uhnsw_exact.restype = C.c_int
    lib.uhnsw_exact.argtypes = [P, P, P, I64, I32, P, P, P]
    lib.uhnsw_idealized_recall.restype = C.c_int
    lib.uhnsw_idealized_recall.argtypes = [P, P, P, I64, I32, I32, C.c_float, P, P]
    lib.uhnsw_plan_t.restype = C.c_int
    lib.uhnsw_plan_t.argtypes = [P, P, I64, I32, I32, C.c_float, C.c_float, C.c_float, I32, P]
    lib.uhnsw_exact_static.restype = C.c_int
    lib.uhnsw_exact_static.argtypes = [P, P, P, I64, I32, P, P, P]
    lib.uhnsw_index_info.restype = C.c_int
    lib.uhnsw_index_info.argtypes = [P, P, P, P, P, P]
    lib.uhnsw_device_status.restype = C.c_int
    lib.uhnsw_device_status.argtypes = [P]
    lib.uhnsw_free.restype = None
    lib.uhnsw_free.argtypes = [P]
    lib.uhnsw_autotune.restype = C.c_int
    lib.uhnsw_autotune.argtypes = [P, P, P, I64, I32, I32, P, P, P, P]
    lib.uhnsw_autotune_save.restype = C.c_int
    lib.uhnsw_autotune_save.argtypes = [P, C.c_char_p]
    lib.uhnsw_autotune_load.restype = C.c_int
    lib.uhnsw_autotune_load.argtypes = [P, C.c_char_p]
    lib.uhnsw_server_create.restype = C.c_int
    lib.uhnsw_server_create.argtypes = [P, P, P]
    lib.uhnsw_server_submit.restype = C.c_int
    lib.uhnsw_server_submit.argtypes = [P, P, C.c_float, I32, I32, P]
    lib.uhnsw_server_poll.restype = C.c_int
    lib.uhnsw_server_poll.argtypes = [P, C.c_uint64, P, P, P]
    lib.uhnsw_server_wait.restype = C.c_int
    lib.uhnsw_server_wait.argtypes = [P, C.c_uint64, P, P, I32]
    lib.uhnsw_server_replay.restype = C.c_int
    lib.uhnsw_server_replay.argtypes = [P, P, P, P, P, I64, P, P, P, P, I32]
    lib.uhnsw_server_stats.restype = C.c_int
    lib.uhnsw_server_stats.argtypes = [P, P]
    lib.uhnsw_server_destroy.restype = None
    lib.uhnsw_server_destroy.argtypes = [P]
    lib.uhnsw_build_graph.restype = C.c_int
    lib.uhnsw_build_graph.argtypes = [P, I64, I32, I32, I32, I32, P, I32, P]
    lib.uhnsw_build_graph_gpu.restype = C.c_int
    lib.uhnsw_build_graph_gpu.argtypes = [P, I64, I32, I32, I32, I32, P, P]
    lib.uhnsw_build_graph_lp.restype = C.c_int
    lib.uhnsw_build_graph_lp.argtypes = [P, I64, I32, C.c_float, I32, I32, P, I32, I32, P]
    lib.uhnsw_probe_sfu.restype = C.c_int
    lib.uhnsw_probe_sfu.argtypes = [I32, I32, P, P, P]
    lib.uhnsw_probe_gather.restype = C.c_int
    lib.uhnsw_probe_gather.argtypes = [P, I64, I32, I32, I32, P, P, P]
    lib.uhnsw_built_graph.restype = C.c_int
    lib.uhnsw_built_graph.argtypes = [P, P]
    lib.uhnsw_built_free.restype = None
    lib.uhnsw_built_free.argtypes = [P]
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise UHNSWError(rc, load_library().uhnsw_last_error().decode(errors="replace"))


def _np_ptr(a) -> C.c_void_p:
    return C.c_void_p(a.ctypes.data) if a is not None else C.c_void_p(0)


def _t_ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream_ptr(stream) -> C.c_void_p:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


# ----------------------------------------------------------------- measurement probes
def probe_sfu(blocks_per_sm: int = 8, iters: int = 4096, stream=None):
    """SFU (lg2 + ex2) rate on the current device: (ms, operations) of one
    timed launch of uhnsw_probe_sfu."""
    ms, ops = C.c_float(0), C.c_double(0)
    _check(load_library().uhnsw_probe_sfu(blocks_per_sm, iters, C.byref(ms), C.byref(ops),
                                          _stream_ptr(stream)))
    return ms.value, ops.value


def probe_gather(buf, row_bytes: int, per_warp: int = 1024, blocks_per_sm: int = 8, stream=None):
    """Random-row gather rate from the device tensor `buf` (its bytes viewed
    as rows of row_bytes): (ms, bytes) of one timed launch of
    uhnsw_probe_gather."""
    rows = buf.numel() * buf.element_size() // row_bytes
    ms, nbytes = C.c_float(0), C.c_double(0)
    _check(load_library().uhnsw_probe_gather(_t_ptr(buf), rows, row_bytes, per_warp,
                                             blocks_per_sm, C.byref(ms), C.byref(nbytes),
                                             _stream_ptr(stream)))
    return ms.value, nbytes.value


# ----------------------------------------------------------------- graph building
def build_graph(base: np.ndarray, metric: int, M: int, ef_construction: int, levels: np.ndarray,
                threads: int = 0, device: str = "cpu", p: float | None = None) -> dict:
    """HNSW graph under L1 (metric=1), squared L2 (metric=2), the L0.5 sum
    (metric=3, U-HNSW-E's G0.5), the L1.5 sum (metric=4) or, with
    metric=BASE_LP and p given, the L_p sum for any 0 < p <= 2, built on the
    host by the library's multi-threaded insertion (device="cpu") or on the
    current CUDA device by batched insertion (device="gpu"); returned as a CSR
    dict {num_levels, entry_point, max_degree0, max_degree, n, levels:
    [{nodes, offsets, nbrs}]} with level 0 listing every node."""
    lib = load_library()
    base = np.ascontiguousarray(base, np.float32)
    levels = np.ascontiguousarray(levels, np.int32)
    n, d = base.shape
    h = C.c_void_p(0)
    if device not in ("cpu", "gpu"):
        raise ValueError(f"device must be 'cpu' or 'gpu', not {device!r}")
    if metric == BASE_LP:
        if p is None:
            raise ValueError("metric BASE_LP needs p")
        _check(lib.uhnsw_build_graph_lp(_np_ptr(base), n, d, float(p), M, ef_construction,
                                        _np_ptr(levels), threads, int(device == "gpu"),
                                        C.byref(h)))
    elif device == "gpu":
        _check(lib.uhnsw_build_graph_gpu(_np_ptr(base), n, d, metric, M, ef_construction,
                                         _np_ptr(levels), C.byref(h)))
    else:
        _check(lib.uhnsw_build_graph(_np_ptr(base), n, d, metric, M, ef_construction,
                                     _np_ptr(levels), threads, C.byref(h)))
    try:
        g = _Graph()
        _check(lib.uhnsw_built_graph(h, C.byref(g)))
        L = g.num_levels
        counts = np.ctypeslib.as_array(C.cast(g.level_count, C.POINTER(C.c_int32)), shape=(L,)).copy()
        out = {"num_levels": L, "entry_point": g.entry_point, "max_degree0": g.max_degree0,
               "max_degree": g.max_degree, "n": n, "levels": []}
        for l in range(L):
            cnt = int(counts[l])
            offs = np.ctypeslib.as_array(C.cast(g.level_offsets[l], C.POINTER(C.c_int64)),
                                         shape=(cnt + 1,)).copy()
            ne = int(offs[-1])
            nbrs = (np.ctypeslib.as_array(C.cast(g.level_nbrs[l], C.POINTER(C.c_int32)),
                                          shape=(ne,)).copy() if ne else np.zeros(0, np.int32))
            if l == 0:
                nodes = np.arange(n, dtype=np.int32)
            else:
                nodes = np.ctypeslib.as_array(C.cast(g.level_nodes[l], C.POINTER(C.c_int32)),
                                              shape=(cnt,)).copy()
            out["levels"].append({"nodes": nodes, "offsets": offs, "nbrs": nbrs})
        return out
    finally:
        lib.uhnsw_built_free(h)


def _graph_struct(g: dict | None):
    if g is None:
        return None, []
    keep = []
    s = _Graph()
    s.num_levels = g["num_levels"]
    s.entry_point = g["entry_point"]
    s.max_degree0 = g["max_degree0"]
    s.max_degree = g["max_degree"]
    cnt = np.array([len(lv["offsets"]) - 1 for lv in g["levels"]], np.int32)
    keep.append(cnt)
    s.level_count = cnt.ctypes.data
    for l, lv in enumerate(g["levels"]):
        nodes = np.ascontiguousarray(lv["nodes"], np.int32)
        offs = np.ascontiguousarray(lv["offsets"], np.int64)
        nbrs = np.ascontiguousarray(lv["nbrs"], np.int32)
        if nbrs.size == 0:
            nbrs = np.zeros(1, np.int32)
        keep += [nodes, offs, nbrs]
        s.level_nodes[l] = nodes.ctypes.data
        s.level_offsets[l] = offs.ctypes.data
        s.level_nbrs[l] = nbrs.ctypes.data
    return s, keep


# ----------------------------------------------------------------- t per p
def plan_t(counts: np.ndarray, p: np.ndarray, K: int, target: float, p_lo: float = 0.5,
           bin_width: float = 0.1, nbins: int = 15) -> np.ndarray:
    """uhnsw_plan_t: the smallest t per p bin whose mean idealized recall reaches
    `target` (bin b holds p in (p_lo + b w, p_lo + (b + 1) w])."""
    counts = np.ascontiguousarray(counts, np.int32)
    p = np.ascontiguousarray(p, np.float32)
    out = np.zeros(nbins, np.int32)
    _check(load_library().uhnsw_plan_t(_np_ptr(counts), _np_ptr(p), counts.shape[0], int(K),
                                       counts.shape[1], float(target), float(p_lo),
                                       float(bin_width), int(nbins), _np_ptr(out)))
    return out


# ----------------------------------------------------------------- index
class Index:
    """A loaded U-HNSW index (base vectors + two graphs) on the current CUDA
    device.  metrics: base metrics of g1 and g2, U_HNSW (G1, G2) by default or
    U_HNSW_E (G0.5, G1; search with cutoff=0.6).  A slot whose metric is
    BASE_LP takes its p from base_p (e.g. metrics=(BASE_LP, BASE_L2),
    base_p=(0.8, 0) for a fixed HNSW under L0.8 beside G2)."""

    def __init__(self, base: np.ndarray, g1: dict | None, g2: dict | None,
                 traverse_dtype: str = "f32", metrics=U_HNSW, base_p=(0.0, 0.0)):
        lib = load_library()
        base = np.ascontiguousarray(base, np.float32)
        self.n, self.d = base.shape
        self.traverse_dtype = traverse_dtype
        s1, k1 = _graph_struct(g1)
        s2, k2 = _graph_struct(g2)
        opts = _LoadOpts()
        opts.traverse_dtype = DTYPES[traverse_dtype]
        opts.base_metric[0], opts.base_metric[1] = int(metrics[0]), int(metrics[1])
        opts.base_p[0], opts.base_p[1] = float(base_p[0]), float(base_p[1])
        self.metrics = tuple(metrics)
        self.base_p = tuple(base_p)
        h = C.c_void_p(0)
        _check(lib.uhnsw_load(_np_ptr(base), self.n, self.d,
                              C.byref(s1) if s1 is not None else None,
                              C.byref(s2) if s2 is not None else None, C.byref(opts), C.byref(h)))
        self._h = h
        del k1, k2

    # -- helpers
    def _opts(self, t=0, kappa=0, tau=0.0, cutoff=0.0, mode="exact", width=1, persistent=False,
              use_graph=False, ef_max=0, stats_t=None, query_threads=0, stage_bytes=0,
              team_lanes=0, hash_bits=0, verify_groups=0):
        o = _SearchOpts()
        o.t, o.kappa, o.tau, o.cutoff = int(t), int(kappa), float(tau), float(cutoff)
        o.verify_mode = MODES[mode] if isinstance(mode, str) else int(mode)
        o.search_width = int(width)
        o.persistent = int(bool(persistent))
        o.use_graph = int(bool(use_graph))
        o.ef_max = int(ef_max)
        o.query_threads = int(query_threads)
        o.stage_bytes = int(stage_bytes)
        o.team_lanes = int(team_lanes)
        o.hash_bits = int(hash_bits)
        o.verify_groups = int(verify_groups)
        o.stats = stats_t.data_ptr() if stats_t is not None else None
        return o

    def search(self, q, p, k=10, ef=64, *, k_max: int | None = None, t=0, tau=0.0,
               kappa: int = 0, cutoff: float = 0.0, mode: str = "exact", width: int = 1,
               persistent: bool = False, use_graph: bool = False, ef_max: int = 0,
               query_threads: int = 0, stage_bytes: int = 0, team_lanes: int = 0,
               hash_bits: int = 0, verify_groups: int = 0,
               stats: bool = False, out=None, stream=None, kernel_events=None):
        """Algorithm 1 on device tensors.  q: float32 [nq, d] cuda; p: float32 [nq];
        k / ef / t: int (same for all) or int32 [nq] tensors; tau: float or
        float32 [nq] tensor.  kernel_events: two
        torch.cuda.Event (already recorded once) bracketing the search kernels
        alone.  Returns (ids int64 [nq, k_max], dist float32 [nq, k_max], stats
        int32 [nq, 8] or None)."""
        import torch
        lib = load_library()
        nq = q.shape[0]
        k_t = k if torch.is_tensor(k) else None
        ef_t = ef if torch.is_tensor(ef) else None
        if k_max is None:
            k_max = int(k_t.max().item()) if k_t is not None and nq else int(k if k_t is None else 1)
        elif k_t is None and int(k) != k_max:
            # one k below the output width: pass it per query (k = NULL means k_max)
            k_t = torch.full((nq,), int(k), dtype=torch.int32, device=q.device)
        ef_default = int(ef) if ef_t is None else max(1, int(ef_max) or MAX_EF)
        if out is None:
            ids = torch.empty((nq, k_max), dtype=torch.int64, device=q.device)
            dist = torch.empty((nq, k_max), dtype=torch.float32, device=q.device)
        else:
            ids, dist = out
        st = torch.zeros((nq, NSTATS), dtype=torch.int32, device=q.device) if stats else None
        t_t = t if torch.is_tensor(t) else None
        tau_t = tau if torch.is_tensor(tau) else None
        o = self._opts(0 if t_t is not None else t, kappa, 0.0 if tau_t is not None else tau,
                       cutoff, mode, width, persistent, use_graph, ef_max, st, query_threads,
                       stage_bytes, team_lanes, hash_bits, verify_groups)
        o.t_per_query = t_t.data_ptr() if t_t is not None else None
        o.tau_per_query = tau_t.data_ptr() if tau_t is not None else None
        if kernel_events is not None:
            evs = (C.c_void_p * 2)(*(int(e.cuda_event) for e in kernel_events))
            if not evs[0] or not evs[1]:
                raise ValueError("kernel_events: record each event once before passing it")
            o.kernel_events = C.cast(evs, C.c_void_p)
        _check(lib.uhnsw_search(self._h, _t_ptr(q), _t_ptr(p), _t_ptr(k_t), _t_ptr(ef_t), nq,
                                k_max, ef_default, C.byref(o), _t_ptr(ids), _t_ptr(dist),
                                _stream_ptr(stream)))
        return ids, dist, st

    def search_host(self, q: np.ndarray, p: np.ndarray, k=10, ef=64, *, k_max: int | None = None,
                    out=None, stream=None, wait: bool = True, **kw):
        """uhnsw_search_host: host (pinned or pageable) arrays in and out.
        wait=False calls uhnsw_search_host_async, which returns once the work
        is queued on `stream`: then `out` must be given, every array must
        already be C-contiguous float32 / int32 (the call makes no temporary
        copies that could be freed before the stream reads them), and none
        may be touched until the stream has synchronised."""
        lib = load_library()
        given = [q, p] + [x for x in (k, ef, kw.get("t"), kw.get("tau")) if isinstance(x, np.ndarray)]
        q = np.ascontiguousarray(q, np.float32)
        p = np.ascontiguousarray(p, np.float32)
        nq = q.shape[0]
        k_a = np.ascontiguousarray(k, np.int32) if isinstance(k, np.ndarray) else None
        ef_a = np.ascontiguousarray(ef, np.int32) if isinstance(ef, np.ndarray) else None
        if k_max is None:
            k_max = int(k_a.max()) if k_a is not None else int(k)
        elif k_a is None and int(k) != k_max:
            if not wait:
                raise ValueError("search_host(wait=False): pass k as an int32 array or k == k_max")
            k_a = np.full(nq, int(k), np.int32)
        if not wait:
            if out is None:
                raise ValueError("search_host(wait=False): `out` must be given")
            used = [q, p] + [x for x in (k_a, ef_a) if x is not None]
            if any(u is not g for u, g in zip(used, given)):
                raise ValueError("search_host(wait=False): arrays must be C-contiguous float32 "
                                 "(q, p) / int32 (k, ef) already")
        ef_default = int(ef) if ef_a is None else max(1, int(kw.get("ef_max", 0)) or MAX_EF)
        if out is None:
            ids = np.empty((nq, k_max), np.int64)
            dist = np.empty((nq, k_max), np.float32)
        else:
            ids, dist = out
        t_in, tau_in = kw.get("t"), kw.get("tau")
        t_a = (np.ascontiguousarray(kw.pop("t"), np.int32)
               if isinstance(kw.get("t"), np.ndarray) else None)
        tau_a = (np.ascontiguousarray(kw.pop("tau"), np.float32)
                 if isinstance(kw.get("tau"), np.ndarray) else None)
        o = self._opts(**{x: kw[x] for x in ("t", "kappa", "tau", "cutoff", "mode", "width",
                                             "persistent", "ef_max", "query_threads",
                                             "stage_bytes", "team_lanes", "hash_bits",
                                             "verify_groups") if x in kw})
        if not wait and any(a is not None and a is not kw_in for a, kw_in in
                            ((t_a, t_in), (tau_a, tau_in))):
            raise ValueError("search_host(wait=False): t / tau arrays must be C-contiguous "
                             "int32 / float32 already")
        o.t_per_query = t_a.ctypes.data if t_a is not None else None
        o.tau_per_query = tau_a.ctypes.data if tau_a is not None else None
        fn = lib.uhnsw_search_host if wait else lib.uhnsw_search_host_async
        _check(fn(self._h, _np_ptr(q), _np_ptr(p), _np_ptr(k_a), _np_ptr(ef_a), nq, k_max,
                  ef_default, C.byref(o), _np_ptr(ids), _np_ptr(dist), _stream_ptr(stream)))
        return ids, dist

    def verify(self, q, p, cand, k: int, *, mode: str = "exact", kappa: int = 0, tau: float = 0.0,
               verify_groups: int = 0, stats: bool = False, stream=None):
        """Verification only on candidate lists cand int32 [nq, t] (-1 = absent)."""
        import torch
        lib = load_library()
        nq, t = cand.shape
        ids = torch.empty((nq, k), dtype=torch.int64, device=q.device)
        dist = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        st = torch.zeros((nq, NSTATS), dtype=torch.int32, device=q.device) if stats else None
        o = self._opts(kappa=kappa, tau=tau, mode=mode, stats_t=st, verify_groups=verify_groups)
        _check(lib.uhnsw_verify(self._h, _t_ptr(q), _t_ptr(p), _t_ptr(cand), t, k, nq, C.byref(o),
                                _t_ptr(ids), _t_ptr(dist), _stream_ptr(stream)))
        return ids, dist, st

    def idealized_recall(self, q, p, K: int, t_max: int, cutoff: float = 0.0, stream=None):
        """uhnsw_idealized_recall: int32 [nq, t_max] tensor of |top-K under L_p of
        each query & top-t under its graph's base metric| for t = 1 .. t_max."""
        import torch
        lib = load_library()
        counts = torch.empty((q.shape[0], t_max), dtype=torch.int32, device=q.device)
        _check(lib.uhnsw_idealized_recall(self._h, _t_ptr(q), _t_ptr(p), q.shape[0], int(K),
                                          int(t_max), float(cutoff), _t_ptr(counts),
                                          _stream_ptr(stream)))
        return counts

    def exact(self, q, p, k: int, stream=None):
        """Exhaustive L_p k-NN on the GPU: (ids int64 [nq, k], dist float32 [nq, k])."""
        import torch
        lib = load_library()
        nq = q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64, device=q.device)
        dist = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        _check(lib.uhnsw_exact(self._h, _t_ptr(q), _t_ptr(p), nq, k, _t_ptr(ids), _t_ptr(dist),
                               _stream_ptr(stream)))
        return ids, dist

    def autotune(self, q, p, k: int, ef: int, stream=None, **base_opts):
        """uhnsw_autotune on a device sample batch: returns (options dict, ms)."""
        lib = load_library()
        b = self._opts(**base_opts)
        best = _SearchOpts()
        ms = C.c_float(0)
        _check(lib.uhnsw_autotune(self._h, _t_ptr(q), _t_ptr(p), q.shape[0], int(k), int(ef),
                                  C.byref(b), _stream_ptr(stream), C.byref(best), C.byref(ms)))
        return ({"query_threads": best.query_threads, "team_lanes": best.team_lanes,
                 "stage_bytes": best.stage_bytes, "hash_bits": best.hash_bits,
                 "verify_groups": best.verify_groups}, ms.value)

    def autotune_save(self, path: str):
        _check(load_library().uhnsw_autotune_save(self._h, path.encode()))

    def autotune_load(self, path: str):
        _check(load_library().uhnsw_autotune_load(self._h, path.encode()))

    def info(self) -> dict:
        lib = load_library()
        n, d, dp, b, m0 = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int64(), C.c_int32()
        _check(lib.uhnsw_index_info(self._h, C.byref(n), C.byref(d), C.byref(dp), C.byref(b),
                                    C.byref(m0)))
        return {"n": n.value, "d": d.value, "d_pad": dp.value, "device_bytes": b.value,
                "max_degree0": m0.value}

    def device_status(self) -> int:
        return load_library().uhnsw_device_status(self._h)

    def close(self):
        if getattr(self, "_h", None):
            load_library().uhnsw_free(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- serving
class _ServerOpts(C.Structure):
    _fields_ = [
        ("max_batch", C.c_int32),
        ("streams", C.c_int32),
        ("state_budget", C.c_int64),
        ("k_max", C.c_int32),
        ("ef_max", C.c_int32),
        ("max_delay_us", C.c_int32),
        ("reserved", C.c_int32),
        ("search", _SearchOpts),
    ]


class _ServerStats(C.Structure):
    _fields_ = [
        ("completed", C.c_int64),
        ("batches", C.c_int64),
        ("mean_batch", C.c_double),
        ("peak_inflight", C.c_int64),
        ("peak_state", C.c_int64),
        ("mean_us", C.c_double),
        ("p50_us", C.c_double),
        ("p99_us", C.c_double),
        ("max_us", C.c_double),
        ("error", C.c_int32),
        ("reserved", C.c_int32),
    ]


class Server:
    """Continuous-batching server over a loaded Index (uhnsw_server_*)."""

    def __init__(self, index: Index, max_batch: int = 1024, streams: int = 4,
                 state_budget: int = 0, k_max: int = 100, ef_max: int = 512,
                 max_delay_us: int = 200, **search_opts):
        lib = load_library()
        o = _ServerOpts()
        o.max_batch, o.streams, o.state_budget = max_batch, streams, state_budget
        o.k_max, o.ef_max, o.max_delay_us = k_max, ef_max, max_delay_us
        o.search = index._opts(**search_opts)
        self.k_max = k_max
        self.index = index
        h = C.c_void_p(0)
        _check(lib.uhnsw_server_create(index._h, C.byref(o), C.byref(h)))
        self._h = h

    def submit(self, q: np.ndarray, p: float, k: int, ef: int) -> int:
        q = np.ascontiguousarray(q, np.float32)
        t = C.c_uint64(0)
        _check(load_library().uhnsw_server_submit(self._h, _np_ptr(q), float(p), int(k), int(ef),
                                                  C.byref(t)))
        return t.value

    def wait(self, ticket: int, k: int, timeout_ms: int = 60000):
        ids = np.empty(k, np.int64)
        dist = np.empty(k, np.float32)
        _check(load_library().uhnsw_server_wait(self._h, ticket, _np_ptr(ids), _np_ptr(dist),
                                                timeout_ms))
        return ids, dist

    def replay(self, q, p, k, ef, arrival_us, timeout_ms: int = 600000):
        """Submit requests at arrival_us (ascending, microseconds) from a native
        thread; returns (ids [nq, k_max], dist [nq, k_max], latency_us [nq])."""
        q = np.ascontiguousarray(q, np.float32)
        nq = q.shape[0]
        p = np.ascontiguousarray(np.broadcast_to(np.asarray(p, np.float32), (nq,)))
        k = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)))
        ef = np.ascontiguousarray(np.broadcast_to(np.asarray(ef, np.int32), (nq,)))
        arr = np.ascontiguousarray(arrival_us, np.float64)
        ids = np.empty((nq, self.k_max), np.int64)
        dist = np.empty((nq, self.k_max), np.float32)
        lat = np.empty(nq, np.float64)
        _check(load_library().uhnsw_server_replay(self._h, _np_ptr(q), _np_ptr(p), _np_ptr(k),
                                                  _np_ptr(ef), nq, _np_ptr(arr), _np_ptr(ids),
                                                  _np_ptr(dist), _np_ptr(lat), timeout_ms))
        return ids, dist, lat

    def stats(self) -> dict:
        st = _ServerStats()
        _check(load_library().uhnsw_server_stats(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_ if f != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            load_library().uhnsw_server_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
