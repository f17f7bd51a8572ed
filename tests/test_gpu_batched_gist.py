"""The batched form on the GIST-shaped workload recipe (d = 960 values in
[0, 1], BF16 traversal copy, FP32 verification), at a reduced N: each query
with its own p, k in {1, 10, 100} and ef in {32 ... 512}, in the bucketed
persistent launch replayed as a CUDA graph.

Float data rounded to BF16 does not let the oracle reproduce the beam id for
id, so the checks are properties that hold at any size: every returned id
carries its own FP64 L_p distance (2e-5 relative), lists are ascending and
duplicate-free, the bucketed persistent launch equals the plain launch bit
for bit, and recall@k against the oracle's exact answer stays high."""
import numpy as np
import pytest

import oracle
from paper_2605_02030_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_gist_shaped_batched_form():
    import paper_2605_02030_gb300 as pkg
    pkg.build()
    from paper_2605_02030_gb300 import uhnsw as U

    w = I.WORKLOADS["gist1m"].scaled(n=12000, nq=48)
    base = I.base_vectors(w)
    qs = I.query_vectors(w)
    p, k, ef = I.query_params(w)
    p[:3] = [1.0, 2.0, 0.5]
    g1 = U.build_graph(base, 1, 16, 100, I.graph_levels(w, 1), threads=0)
    g2 = U.build_graph(base, 2, 16, 100, I.graph_levels(w, 2), threads=0)
    idx = U.Index(base, g1, g2, traverse_dtype="bf16")
    q, pp, kk, ee = (torch.from_numpy(a).cuda() for a in (qs, p, k, ef))
    a = idx.search(q, pp, k=kk, ef=ee, k_max=100, ef_max=512, stats=True)
    b = idx.search(q, pp, k=kk, ef=ee, k_max=100, ef_max=512, persistent=True, use_graph=True)
    torch.cuda.synchronize()
    assert idx.device_status() == 0
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    ids, dist, st = a[0].cpu().numpy(), a[1].cpu().numpy(), a[2].cpu().numpy()
    assert (st[:, 5] == 0).all()
    gt, _ = oracle.exact_knn(base, qs, p, 100)
    hits = total = 0
    for i in range(w.nq):
        ki = int(k[i])
        got = ids[i, :ki]
        assert (got >= 0).all() and len(set(got.tolist())) == ki
        assert (ids[i, ki:] == -1).all()
        ref = np.array([oracle.lp_sum(base[j], qs[i], float(p[i])) ** (1 / float(p[i])) for j in got])
        np.testing.assert_allclose(dist[i, :ki], ref, rtol=2e-5, err_msg=f"query {i}")
        assert np.all(np.diff(dist[i, :ki]) >= -2e-5 * dist[i, 1:ki])
        hits += len(set(got.tolist()) & set(gt[i, :ki].tolist()))
        total += ki
    assert hits / total >= 0.9
    idx.close()
