"""Several expansions per step (`search_width`, the fast mode): the beam
takes the first `width` unexpanded entries of W as parents of one step.  On
0/1 data every base distance is an exact integer in FP32 (and the FP16 copy
is exact), so the GPU beam equals the oracle's width-w search id for id, and
Algorithm 1 on top of it equals the oracle's, in both search kernels."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def binary_case():
    r = np.random.default_rng(41)
    base = r.integers(0, 2, size=(3000, 32)).astype(np.float32)
    qs = r.integers(0, 2, size=(36, 32)).astype(np.float32)
    g1 = oracle.hnsw_build(base, 1, 8, 40, I.hnsw_levels(len(base), 8, 3))
    g2 = oracle.hnsw_build(base, 2, 8, 40, I.hnsw_levels(len(base), 8, 4))
    return base, qs, g1, g2


@pytest.mark.parametrize("width", [2, 3, 5])
@pytest.mark.parametrize("qt", [32, 128])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_wide_beam_equals_oracle(U, binary_case, width, qt, dtype):
    base, qs, g1, g2 = binary_case
    idx = U.Index(base, g1, g2, traverse_dtype=dtype)
    p = np.resize(np.array([1.0, 2.0, 0.6, 1.3, 1.7, 0.9], np.float32), len(qs))
    ids, dist, st = idx.search(dev(qs), dev(p), k=10, ef=32, width=width, query_threads=qt,
                               stats=True)
    ids, dist, st = ids.cpu().numpy(), dist.cpu().numpy(), st.cpu().numpy()
    for i in range(len(qs)):
        rid, rd, _ = oracle.uhnsw_query(g1, g2, base, qs[i], float(p[i]), 10, 32, width=width)
        np.testing.assert_array_equal(ids[i], rid, err_msg=f"query {i} p={p[i]}")
        np.testing.assert_allclose(dist[i], rd, rtol=2e-5, err_msg=f"query {i} p={p[i]}")
    assert (st[:, 5] == 0).all()
    assert idx.device_status() == 0
    idx.close()


@pytest.mark.parametrize("width", [2, 4])
def test_wide_beam_persistent_graph_replay(U, binary_case, width):
    """The batched form (persistent queue, CUDA-graph replay) returns what
    the plain launch returns at the same width."""
    base, qs, g1, g2 = binary_case
    idx = U.Index(base, g1, g2, traverse_dtype="f16")
    p = np.resize(np.array([0.7, 1.0, 1.5, 2.0], np.float32), len(qs))
    a = idx.search(dev(qs), dev(p), k=10, ef=40, width=width)
    b = idx.search(dev(qs), dev(p), k=10, ef=40, width=width, persistent=True, use_graph=True)
    c = idx.search(dev(qs), dev(p), k=10, ef=40, width=width, persistent=True, use_graph=True)
    for x, y in ((a, b), (b, c)):
        assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1])
    idx.close()
