"""uhnsw_exact_static: exhaustive L_p k-NN without allocating device memory.

Callers on a fixed, pre-reserved memory budget (a serving loop), callers whose
device memory belongs to another framework's caching allocator, and
latency-critical code that must not hit the device-wide synchronisation of
cudaMalloc / cudaFree cannot use uhnsw_exact, which grows its workspace on
demand.  uhnsw_exact_static keeps that workspace in a fixed device array
instead.  This test calls both entry points through the C ABI and checks, on
two calls in a row, that the allocation-free one returns the oracle's exact
FP64 answer and the same answer as uhnsw_exact (the array keeps the previous
call's contents, which must not leak into the next).
The file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle

from helpers import check_topk, oracle_graphs, workload_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_exact_static_matches_exact_twice():
    import paper_2605_02030_gb300 as pkg
    pkg.build()
    from paper_2605_02030_gb300 import uhnsw as U

    lib = U.load_library()
    w, base, qs, p, _, _ = workload_arrays("sift1m", 3000, 48)
    g1, g2 = oracle_graphs("sift1m", 3000, 24, M=8, ef_construction=40)
    idx = U.Index(base, g1, g2)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    k = 10
    # two different query batches: the second must not see the first one's scratch
    for lo, hi in ((0, 48), (8, 40)):
        q = torch.from_numpy(qs[lo:hi]).cuda()
        pv = torch.from_numpy(p[lo:hi]).cuda()
        nq = hi - lo
        ids_a = torch.full((nq, k), -7, dtype=torch.int64, device="cuda")
        dist_a = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
        ids_b = torch.full((nq, k), -7, dtype=torch.int64, device="cuda")
        dist_b = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
        rc = lib.uhnsw_exact(idx._h, _ptr(q), _ptr(pv), nq, k, _ptr(ids_a), _ptr(dist_a), stream)
        assert rc == 0, lib.uhnsw_last_error()
        rc = lib.uhnsw_exact_static(idx._h, _ptr(q), _ptr(pv), nq, k, _ptr(ids_b), _ptr(dist_b),
                                    stream)
        assert rc == 0, lib.uhnsw_last_error()
        torch.cuda.synchronize()
        a_ids, a_d = ids_a.cpu().numpy(), dist_a.cpu().numpy()
        b_ids, b_d = ids_b.cpu().numpy(), dist_b.cpu().numpy()
        ref_ids, _ = oracle.exact_knn(base, qs[lo:hi], p[lo:hi], k)
        for i in range(nq):
            # the same tolerance rule as every parity test: ids equal to the
            # oracle's exact top-k except near-ties, distances within 2e-5 of
            # the FP64 oracle; and the allocating entry point agrees
            check_topk(base, qs[lo + i], p[lo + i], b_ids[i], b_d[i], ref_ids[i], k,
                       f"static q{lo + i}")
            check_topk(base, qs[lo + i], p[lo + i], b_ids[i], b_d[i], a_ids[i], k,
                       f"static vs uhnsw_exact q{lo + i}")
        np.testing.assert_allclose(b_d, a_d, rtol=2e-5)
    # a request larger than the fixed array is refused before any work
    big = 32 * 1024 * 1024 // (8 * k) + 1
    rc = lib.uhnsw_exact_static(idx._h, _ptr(q), _ptr(pv), big, k, _ptr(ids_b), _ptr(dist_b),
                                stream)
    assert rc == -5 and b"exceeds" in lib.uhnsw_last_error()
    assert idx.device_status() == 0
    idx.close()
