"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only draws random numbers with the distributions of the
workloads below; it holds none of the query method's arithmetic (no
distance, no search, no verification).  Every draw comes from a
``numpy.random.default_rng`` stream (PCG64), whose output does not depend
on the host architecture, so x86 and Arm hosts produce identical arrays.

Streams for a workload with seed ``s``:
  s     base vectors
  s+1   query vectors
  s+2   per-query p, k and ef
  s+3   HNSW levels of the L1 graph (G1)
  s+4   HNSW levels of the L2 graph (G2)
  s+5   HNSW levels of the L0.5 graph (G0.5, U-HNSW-E)
  s+6   held-out calibration query vectors (drawn like the queries)
  s+7   held-out calibration p, k and ef (drawn like the query parameters)

The HNSW level of each node is a random draw of the index construction
(level = floor(-ln(U) * mL), mL = 1/ln(M), U uniform in (0, 1]); it is drawn
here and passed to both graph builders as an input.

Workloads (synthetic stand-ins for the paper's datasets, Table 1; no
dataset item is reproduced):
  mixture10k   N=10,000 d=32 Gaussian mixture, 16 centres ~ N(0, 4I),
               points = centre + N(0, I); 100 queries from the mixture;
               p ~ U(0.5, 2]; k=10; M=16, efConstruction=100; ef=64.
  sift1m       N=1,000,000 d=128 integer features 0..255 (SIFT-shaped):
               1,000 centres with per-dimension Exp(mean 30) clipped to
               [0, 255]; x = round(clip(centre + N(0, 20^2), 0, 255));
               10,000 queries from the same generator; p on the grid
               {0.5, 0.6, ..., 2.0}; k=10; M=32, efConstruction=200.
  sift1m_fp16  sift1m's base and queries, p ~ U(0.5, 2]; the traversal copy
               is FP16 (0..255 is exact in FP16).
  gist1m       N=1,000,000 d=960 in [0, 1] (GIST-shaped): 100 clusters,
               centre mu ~ Beta(2, 5) per dimension, x ~ Beta(20 mu,
               20 (1 - mu)); p ~ U(0.5, 2]; k in {1, 10, 100}; ef in
               {32, 64, 128, 256, 512} with ef >= k; BF16 traversal copy.
               Its rows are drawn in blocks of 16,384, block i from child i
               of a seed drawn from the workload's stream.
  unit10m      N=10,000,000 d=96 N(0, I) rows scaled to unit L2 norm, FP16;
               p ~ U(0.5, 2]; k in {10, 50}.
  sift1m_e     sift1m's base and queries for U-HNSW-E (Section 4.5): graphs
               under L0.5 and L1, cutoff 0.6, p ~ U(0.2, 0.7] (the shifted
               range of the paper's comparison); FP16 traversal copy.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field, replace

import numpy as np

P_GRID = np.round(np.arange(0.5, 2.0 + 1e-9, 0.1), 1).astype(np.float32)  # 16 values


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    nq: int
    kind: str               # "mixture" | "sift" | "gist" | "unit"
    p_mode: str             # "uniform" | "grid"
    k: int = 10
    k_choices: tuple = ()
    ef: int = 64
    ef_choices: tuple = ()
    M: int = 16
    ef_construction: int = 100
    n_clusters: int = 16
    traverse_dtype: str = "f32"
    p_lo: float = 0.5       # "uniform" p is drawn on (p_lo, p_hi]
    p_hi: float = 2.0
    metrics: tuple = (1, 2)  # base metrics of the two graphs (3 = L0.5)
    cutoff: float = 1.4
    seed: int = 0
    grid: float = 0.0       # >0: round base and queries to multiples of `grid`
    extra: dict = field(default_factory=dict)

    def scaled(self, n: int | None = None, nq: int | None = None, **kw) -> "Workload":
        """Same recipe at another size (smaller parity cases)."""
        return replace(self, n=self.n if n is None else n, nq=self.nq if nq is None else nq, **kw)


WORKLOADS = {
    "mixture10k": Workload("mixture10k", 10_000, 32, 100, "mixture", "uniform", k=10, ef=64,
                           M=16, ef_construction=100, n_clusters=16),
    "sift1m": Workload("sift1m", 1_000_000, 128, 10_000, "sift", "grid", k=10, ef=64,
                       ef_choices=(16, 32, 64, 128, 256, 512), M=32, ef_construction=200,
                       n_clusters=1000),
    "sift1m_fp16": Workload("sift1m_fp16", 1_000_000, 128, 10_000, "sift", "uniform", k=10, ef=64,
                            ef_choices=(16, 32, 64, 128, 256, 512), M=32, ef_construction=200,
                            n_clusters=1000, traverse_dtype="f16"),
    "gist1m": Workload("gist1m", 1_000_000, 960, 10_000, "gist", "uniform", k=10,
                       k_choices=(1, 10, 100), ef=128, ef_choices=(32, 64, 128, 256, 512),
                       M=32, ef_construction=200, n_clusters=100, traverse_dtype="bf16"),
    "unit10m": Workload("unit10m", 10_000_000, 96, 10_000, "unit", "uniform", k=10,
                        k_choices=(10, 50), ef=128, M=32, ef_construction=200,
                        traverse_dtype="f16"),
    "sift1m_e": Workload("sift1m_e", 1_000_000, 128, 10_000, "sift", "uniform", k=10, ef=64,
                         M=32, ef_construction=200, n_clusters=1000, traverse_dtype="f16",
                         p_lo=0.2, p_hi=0.7, metrics=(3, 1), cutoff=0.6),
}


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def _mixture(rng: np.random.Generator, centres: np.ndarray, n: int, point_std: float) -> np.ndarray:
    c = rng.integers(0, centres.shape[0], size=n)
    x = centres[c] + rng.standard_normal((n, centres.shape[1]), dtype=np.float32) * point_std
    return x.astype(np.float32)


def _centres(w: Workload) -> np.ndarray:
    """Cluster centres, drawn from the base stream's own generator (seed 1000+seed)."""
    rng = _rng(1000 + w.seed)
    if w.kind == "mixture":
        return (rng.standard_normal((w.n_clusters, w.d), dtype=np.float32) * 2.0).astype(np.float32)
    if w.kind == "sift":
        return np.clip(rng.exponential(30.0, size=(w.n_clusters, w.d)), 0, 255).astype(np.float32)
    if w.kind == "gist":
        return rng.beta(2.0, 5.0, size=(w.n_clusters, w.d)).astype(np.float32)
    raise ValueError(w.kind)


def _draw_points(w: Workload, rng: np.random.Generator, n: int, centres) -> np.ndarray:
    if w.kind == "mixture":
        x = _mixture(rng, centres, n, 1.0)
    elif w.kind == "sift":
        x = np.empty((n, w.d), dtype=np.float32)
        step = 65536
        for s in range(0, n, step):
            m = min(step, n - s)
            c = rng.integers(0, centres.shape[0], size=m)
            v = centres[c] + rng.standard_normal((m, w.d), dtype=np.float32) * 20.0
            x[s:s + m] = np.rint(np.clip(v, 0.0, 255.0))
    elif w.kind == "gist":
        # Beta draws are slow: each block of 16,384 rows has a stream of its
        # own (child i of the stream's seed), so the blocks are drawn on
        # several threads and the array does not depend on their number
        x = np.empty((n, w.d), dtype=np.float32)
        step = 16384
        seed = int(rng.integers(0, 2 ** 63))

        def block(i):
            s = i * step
            m = min(step, n - s)
            r = np.random.default_rng(np.random.SeedSequence(seed, spawn_key=(i,)))
            c = r.integers(0, centres.shape[0], size=m)
            mu = np.clip(centres[c], 1e-3, 1 - 1e-3)
            x[s:s + m] = r.beta(20.0 * mu, 20.0 * (1.0 - mu)).astype(np.float32)

        nblocks = (n + step - 1) // step
        with ThreadPoolExecutor(max_workers=max(1, min(nblocks, os.cpu_count() or 1))) as ex:
            list(ex.map(block, range(nblocks)))
    elif w.kind == "unit":
        x = np.empty((n, w.d), dtype=np.float32)
        step = 1 << 18
        for s in range(0, n, step):
            m = min(step, n - s)
            v = rng.standard_normal((m, w.d), dtype=np.float32)
            x[s:s + m] = v / np.linalg.norm(v, axis=1, keepdims=True)
    else:
        raise ValueError(w.kind)
    if w.grid > 0:
        x = (np.rint(x / w.grid) * w.grid).astype(np.float32)
    return np.ascontiguousarray(x, dtype=np.float32)


def base_vectors(w: Workload) -> np.ndarray:
    """Base set D, float32 [n, d] row-major."""
    centres = None if w.kind == "unit" else _centres(w)
    return _draw_points(w, _rng(w.seed), w.n, centres)


def query_vectors(w: Workload) -> np.ndarray:
    """Query vectors, float32 [nq, d], drawn like the base set."""
    centres = None if w.kind == "unit" else _centres(w)
    return _draw_points(w, _rng(w.seed + 1), w.nq, centres)


def query_params(w: Workload, stream: int = 2):
    """Per-query (p float32 [nq], k int32 [nq], ef int32 [nq]) from stream
    seed + `stream` (2: the queries; 7: the held-out calibration set)."""
    rng = _rng(w.seed + stream)
    if w.p_mode == "grid":
        p = P_GRID[rng.integers(0, len(P_GRID), size=w.nq)]
    else:
        # uniform on (p_lo, p_hi]: p_hi - (p_hi - p_lo) U with U uniform on [0, 1)
        p = (w.p_hi - (w.p_hi - w.p_lo) * rng.random(w.nq)).astype(np.float32)
    if w.k_choices:
        k = np.asarray(w.k_choices, dtype=np.int32)[rng.integers(0, len(w.k_choices), size=w.nq)]
    else:
        k = np.full(w.nq, w.k, dtype=np.int32)
    if w.ef_choices:
        ef = np.asarray(w.ef_choices, dtype=np.int32)[rng.integers(0, len(w.ef_choices), size=w.nq)]
        ef = np.maximum(ef, k).astype(np.int32)
    else:
        ef = np.full(w.nq, w.ef, dtype=np.int32)
    return p.astype(np.float32), k, ef


def calibration_set(w: Workload):
    """A held-out query set of the same recipe and size as the workload's
    queries, from streams of its own: (vectors float32 [nq, d], p, k, ef).
    A search's beam can be chosen on it and its recall then reported on the
    workload's own queries."""
    centres = None if w.kind == "unit" else _centres(w)
    q = _draw_points(w, _rng(w.seed + 6), w.nq, centres)
    p, k, ef = query_params(w, stream=7)
    return q, p, k, ef


def p_bin_edges(w: Workload, nbins: int = 16) -> np.ndarray:
    """Upper edges of `nbins` equal p bins on (p_lo, p_hi] (uniform p), or the
    grid values themselves (grid p)."""
    if w.p_mode == "grid":
        return P_GRID.copy()
    return (w.p_lo + (w.p_hi - w.p_lo) * np.arange(1, nbins + 1) / nbins).astype(np.float64)


def p_bin_of(w: Workload, p: np.ndarray, nbins: int = 16) -> np.ndarray:
    """Bin index of each p: on the grid, the grid value's position; for
    uniform p on (lo, hi], bin b holds (lo + b h, lo + (b + 1) h], h = (hi -
    lo) / nbins."""
    p = np.asarray(p, np.float64)
    if w.p_mode == "grid":
        return np.clip(np.rint((p - float(P_GRID[0])) / 0.1).astype(int), 0, len(P_GRID) - 1)
    h = (w.p_hi - w.p_lo) / nbins
    return np.clip(np.ceil((p - w.p_lo) / h - 1e-9).astype(int) - 1, 0, nbins - 1)


def hnsw_levels(n: int, M: int, seed: int) -> np.ndarray:
    """Random HNSW layer of each node: floor(-ln(U) / ln(M)), U uniform on (0, 1]."""
    rng = _rng(seed)
    u = 1.0 - rng.random(n)              # (0, 1]
    lv = np.floor(-np.log(u) / math.log(M)).astype(np.int32)
    return np.minimum(lv, 15).astype(np.int32)


def graph_levels(w: Workload, metric: int) -> np.ndarray:
    """Levels for G1 (metric=1), G2 (metric=2) or G0.5 (metric=3) of workload `w`."""
    return hnsw_levels(w.n, w.M, w.seed + {1: 3, 2: 4, 3: 5}[metric])


def random_candidates(n: int, nq: int, t: int, seed: int, missing_frac: float = 0.0) -> np.ndarray:
    """Candidate id lists [nq, t] int32 drawn without replacement per row;
    a fraction of trailing slots is set to -1 (absent) when asked."""
    rng = _rng(seed)
    out = np.empty((nq, t), dtype=np.int32)
    for i in range(nq):
        out[i] = rng.choice(n, size=t, replace=False)
    if missing_frac > 0:
        cut = rng.integers(int(t * (1 - missing_frac)), t + 1, size=nq)
        for i in range(nq):
            out[i, cut[i]:] = -1
    return out
