"""GPU parity of the graph-diffusion path (Sec. 3.3, Eq. 7 / Eq. 8) against the
CPU oracle, through the C ABI: kNN and the union edge set bit-exact, edge
weights and diffusion within float32 error of the float64 oracle (1e-5 after
one step, 1e-4 after 100 steps, relative L2)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_14462_gb300 import inputs, ludvig
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2410_14462_gb300 import build
    build.build()
    ludvig.load()


def _scene(n, seed):
    return inputs.scene_clusters(n, seed=seed, n_clusters=12, sigma=0.1, extent=1.0)


@pytest.mark.parametrize("n,k", [(20_000, 16), (3000, 5), (1000, 64)])
def test_knn_bitexact(n, k):
    s = _scene(n, 2)
    sc = ludvig.Scene.from_inputs(s)
    got = ludvig.knn(sc, k).cpu().numpy()
    ref, _ = oracle.knn(s.means, k)
    assert np.array_equal(got, ref)


def test_knn_duplicates_and_tiny():
    means = np.zeros((6, 3), np.float32)
    means[3:] = 1.0
    s = inputs.Scene(means, np.ones((6, 3), np.float32) * 0.01,
                     np.tile(np.array([1, 0, 0, 0], np.float32), (6, 1)), np.full(6, 0.5, np.float32))
    sc = ludvig.Scene.from_inputs(s)
    got = ludvig.knn(sc, 8).cpu().numpy()
    ref, _ = oracle.knn(means, 8)
    assert np.array_equal(got, ref)


def _features(n, df, seed):
    rng = np.random.default_rng(seed)
    f = rng.normal(size=(n, df)).astype(np.float32)
    f[::97] = 0.0   # zero vectors: cosine 0
    return f


@pytest.mark.parametrize("row_normalize", [True, False])
def test_graph_matches_oracle(row_normalize):
    n, k, df = 8000, 16, 24
    s = _scene(n, 3)
    f = _features(n, df, 4)
    sc = ludvig.Scene.from_inputs(s)
    g = ludvig.Graph(sc, k, torch.from_numpy(f).cuda(), spatial_h=0.01, row_normalize=row_normalize)
    rp, col, val = (t.cpu().numpy() for t in g.export())
    nbr, _ = oracle.knn(s.means, k)
    rows, cols = oracle.union_edges(nbr)
    assert g.nnz == rows.size
    got_rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.array_equal(got_rows, rows) and np.array_equal(col, cols)
    w = oracle.edge_weights_spatial_cos(s.means, f, rows, cols, h=0.01)
    A = oracle.csr(n, rows, cols, w, row_normalize=row_normalize)
    ref = np.asarray(A[rows, cols]).ravel()
    e = rel_l2(val, ref)
    print(f"edge weights rel L2 {e:.2e}")
    assert e <= 1e-5


def test_diffusion_matches_oracle():
    n, k, df = 20_000, 16, 32
    s = _scene(n, 5)
    f = _features(n, df, 6)
    sc = ludvig.Scene.from_inputs(s)
    g = ludvig.Graph(sc, k, torch.from_numpy(f).cuda(), spatial_h=0.01)
    nbr, _ = oracle.knn(s.means, k)
    rows, cols = oracle.union_edges(nbr)
    A = oracle.csr(n, rows, cols, oracle.edge_weights_spatial_cos(s.means, f, rows, cols, 0.01))
    x0 = (np.linalg.norm(s.means - s.means[0], axis=1) < 0.15).astype(np.float32)
    xt = torch.from_numpy(x0).cuda()
    for iters, tol in [(1, 1e-5), (7, 1e-5), (100, 1e-4)]:
        got = g.diffuse(xt, iters).cpu().numpy()
        ref = oracle.diffuse(A, x0, iters)
        e = rel_l2(got, ref)
        print(f"diffusion {iters} steps rel L2 {e:.2e}")
        assert e <= tol
    # multi-query (several columns) and a zero column
    X = np.stack([x0, np.zeros(n, np.float32), (s.means[:, 0] > 0).astype(np.float32)], 1)
    got = g.diffuse(torch.from_numpy(X).cuda(), 10).cpu().numpy()
    ref = oracle.diffuse(A, X, 10)
    assert rel_l2(got, ref) <= 1e-5
    assert (got[:, 1] == 0).all()
    assert np.array_equal(g.diffuse(xt, 0).cpu().numpy(), x0)


def test_diffusion_resumes_from_an_intermediate_state():
    """Eq. 8 depends only on g_t, so 2 steps then 5 more equal 7 steps at once
    (checkpoint / resume of the diffusion), for one and for several columns."""
    wl = inputs.small_field_workload(n=20_000, views=1, d=16)
    sc = ludvig.Scene.from_inputs(wl.scene)
    f = np.random.default_rng(1).normal(size=(sc.n, 16)).astype(np.float32)
    g = ludvig.Graph(sc, 16, torch.from_numpy(f).cuda(), spatial_h=0.01)
    for dx in (1, 3):
        x0 = torch.rand((sc.n, dx) if dx > 1 else (sc.n,), device="cuda",
                        generator=torch.Generator("cuda").manual_seed(dx))
        whole = g.diffuse(x0, 7)
        part = g.diffuse(g.diffuse(x0, 2), 5)
        torch.cuda.synchronize()
        assert rel_l2(part.cpu().numpy(), whole.cpu().numpy()) <= 1e-6
