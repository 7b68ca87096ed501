"""ludvig_diffuse_noalloc: the graph diffusion for callers that must not
allocate device memory (a warm request loop under a no-allocation policy, a
process whose device memory belongs to another allocator).  Its scratch is the
library's static device memory, so the call is checked against the
allocating ludvig_diffuse on the same inputs, twice in a row (the second call
must not see the first call's leftovers), for one and for several columns; a
warm call leaves the device's free memory, torch's pool and the graph's
workspace unchanged; and its size limit is checked.  Collected last on
purpose: the file name sorts after every other test file."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2410_14462_gb300 import inputs, ludvig

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graph():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2410_14462_gb300 import build
    build.build()
    ludvig.load()
    s = inputs.scene_clusters(20_000, seed=7, n_clusters=10, sigma=0.1, extent=1.0)
    f = np.random.default_rng(7).normal(size=(s.n, 16)).astype(np.float32)
    sc = ludvig.Scene.from_inputs(s)
    g = ludvig.Graph(sc, 16, torch.from_numpy(f).cuda(), spatial_h=0.01)
    return s, sc, g


def _rel(a, b):
    return float((a - b).norm() / max(b.norm().item(), 1e-30))


def test_noalloc_matches_allocating_call_twice(graph):
    s, sc, g = graph
    x0 = torch.from_numpy((np.linalg.norm(s.means - s.means[0], axis=1) < 0.2).astype(np.float32)).cuda()
    x1 = torch.from_numpy((s.means[:, 0] > 0.3).astype(np.float32)).cuda()
    for x, iters in ((x0, 100), (x1, 7)):       # two calls in a row, different inputs
        ref = g.diffuse(x, iters)
        got = torch.full_like(x, float("nan"))
        g.diffuse_noalloc(x, iters, got)
        torch.cuda.synchronize()
        e = _rel(got, ref)
        print(f"single column, {iters} steps: rel L2 vs ludvig_diffuse {e:.2e}")
        assert e <= 1e-5
    X = torch.stack([x0, torch.zeros_like(x0), x1], 1).contiguous()
    for _ in range(2):
        ref = g.diffuse(X, 12)
        got = torch.empty_like(X)
        g.diffuse_noalloc(X, 12, got)
        torch.cuda.synchronize()
        assert _rel(got, ref) <= 1e-5
        assert (got[:, 1] == 0).all()


def test_noalloc_warm_call_allocates_nothing(graph):
    s, sc, g = graph
    x = torch.from_numpy((s.means[:, 1] > 0.0).astype(np.float32)).cuda()
    X = torch.stack([x, 1.0 - x], 1).contiguous()
    out, OUT = torch.empty_like(x), torch.empty_like(X)
    g.diffuse_noalloc(x, 20, out)                      # first call: kernels loaded, nothing else
    g.diffuse_noalloc(X, 20, OUT)
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved(), g.workspace_bytes(),
              sc.workspace_bytes())
    for _ in range(3):
        g.diffuse_noalloc(x, 20, out)
        g.diffuse_noalloc(X, 20, OUT)
    torch.cuda.synchronize()
    after = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved(), g.workspace_bytes(),
             sc.workspace_bytes())
    print(f"free bytes, torch reserved, graph and scene workspace: {before} -> {after}")
    assert after == before


def test_noalloc_rejects_sizes_beyond_its_scratch(graph):
    s, sc, g = graph
    L = ludvig.load()
    x = torch.zeros((s.n, 32), device="cuda")        # 640k elements: within the limit
    out = torch.empty_like(x)
    g.diffuse_noalloc(x, 3, out)
    rc = L.ludvig_diffuse_noalloc(g._h, ctypes.c_void_p(x.data_ptr()), 32, 5000,
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1 and b"iters" in L.ludvig_last_error()
    # 40k nodes x 32 columns = 1.28M elements: beyond the static scratch
    s2 = inputs.scene_clusters(40_000, seed=8, n_clusters=10, sigma=0.1, extent=1.0)
    sc2 = ludvig.Scene.from_inputs(s2)
    g2 = ludvig.Graph(sc2, 4, torch.ones((s2.n, 4), device="cuda"), spatial_h=0.01)
    x2 = torch.zeros((s2.n, 32), device="cuda")
    o2 = torch.empty_like(x2)
    rc = L.ludvig_diffuse_noalloc(g2._h, ctypes.c_void_p(x2.data_ptr()), 32, 3,
                                  ctypes.c_void_p(o2.data_ptr()), None)
    assert rc == 1 and b"exceeds" in L.ludvig_last_error()
    g2.diffuse_noalloc(x2[:, :16].contiguous(), 3, torch.empty((s2.n, 16), device="cuda"))   # 640k: fits
    torch.cuda.synchronize()
