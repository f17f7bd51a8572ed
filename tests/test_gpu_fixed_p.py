"""Fixed-p HNSW (Section 4.3's comparison): a graph built under the query's
own metric answers that p directly.  Here the L1.5 graph (metric 4): on 0/1
data every |d_j|^(3/2) is exactly 0 or 1, so the GPU beam of a p = 1.5 query
equals the oracle's search on the same graph id for id, and the GPU-built
L1.5 graph keeps HNSW's structure."""
import numpy as np
import pytest

import oracle
from paper_2605_02030_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    import paper_2605_02030_gb300 as pkg
    pkg.build()
    from paper_2605_02030_gb300 import uhnsw
    uhnsw.load_library()
    return uhnsw


@pytest.mark.parametrize("qt", [32, 128])
def test_direct_p15_beam_equals_oracle(U, qt):
    r = np.random.default_rng(23)
    base = r.integers(0, 2, size=(2500, 32)).astype(np.float32)
    qs = r.integers(0, 2, size=(30, 32)).astype(np.float32)
    g15 = oracle.hnsw_build(base, 4, 8, 40, I.hnsw_levels(len(base), 8, 6))
    g2 = oracle.hnsw_build(base, 2, 8, 40, I.hnsw_levels(len(base), 8, 4))
    idx = U.Index(base, g15, g2, traverse_dtype="f16", metrics=(U.BASE_L15, U.BASE_L2))
    ef = 24
    p = np.full(len(qs), 1.5, np.float32)
    ids, dist, st = idx.search(torch.from_numpy(qs).cuda(), torch.from_numpy(p).cuda(), k=ef,
                               ef=ef, query_threads=qt, stats=True)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    for i in range(len(qs)):
        rid, rd, _ = oracle.hnsw_search(g15, base, qs[i], 4, ef, ef)
        np.testing.assert_array_equal(ids[i], rid, err_msg=f"query {i}")
        np.testing.assert_allclose(dist[i], rd ** (1 / 1.5), rtol=2e-6)
    assert (st[:, 6] == 1).all() and (st[:, 1] == 0).all()
    idx.close()


def test_gpu_built_l15_graph_structure(U):
    r = np.random.default_rng(24)
    base = r.normal(size=(3000, 48)).astype(np.float32)
    lv = I.hnsw_levels(len(base), 8, 6)
    g = U.build_graph(base, 4, 8, 40, lv, device="gpu")
    assert g["num_levels"] == lv.max() + 1 and lv[g["entry_point"]] == lv.max()
    for l, L in enumerate(g["levels"]):
        assert np.diff(L["offsets"]).max() <= (16 if l == 0 else 8)
        assert (lv[L["nbrs"]] >= l).all()
