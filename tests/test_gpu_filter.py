"""GPU parity of Gaussian filtering (Sec. 3.2, "Gaussian filtering") through
the C ABI: ludvig_beta_select is bit-exact against the oracle's selection on
the same beta values (ties, NaN, non-positive values, sizes spanning several
sort tiles with a ragged tail, every keep edge case); ludvig_scene_subset gives
a scene that projects bit-exactly like the oracle's subset and uplifts within
the float32 bar (1e-5 relative L2); an out-of-range index is an argument
error found by the gather's own bounds check."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_14462_gb300 import inputs, ludvig
from tests.gpu_util import device_features, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2410_14462_gb300 import build
    build.build()
    ludvig.load()


def _scene_of_size(n, seed=0):
    return ludvig.Scene.from_inputs(inputs.scene_uniform(n, seed=seed))


@pytest.mark.parametrize("n", [1, 7, 3 * 4096 + 123])
def test_select_bitexact_with_ties(n):
    sc = _scene_of_size(n)
    rng = np.random.default_rng(n)
    beta = rng.choice(np.array([0.0, 0.125, 0.5, 0.5, 2.0, -1.0, np.nan], np.float32), size=n)
    cont = rng.random(n) < 0.3
    beta[cont] = rng.random(int(cont.sum())).astype(np.float32)
    bt = torch.from_numpy(beta).cuda()
    for keep in sorted({1, n // 2, n - n // 2, max(n - 1, 1), n}):
        got = ludvig.beta_select(sc, bt, keep).cpu().numpy()
        ref = oracle.beta_select(beta, keep)
        assert np.array_equal(got, ref), (n, keep)
    assert ludvig.beta_select(sc, bt, 0).numel() == 0


def test_filter_uplift_pipeline_matches_oracle():
    wl = inputs.small_field_workload(n=20_000, views=3, d=48, width=100, height=75)
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = device_features(wl, range(3))
    out, beta = ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, F)
    torch.cuda.synchronize()
    b = beta.cpu().numpy()
    keep = sc.n - sc.n // 2
    kept = ludvig.beta_select(sc, beta, keep)
    k = kept.cpu().numpy()
    assert np.array_equal(k, oracle.beta_select(b, keep)), "selection differs on the same beta"
    sub = sc.subset(kept)
    ref_scene = wl.scene.subset(k)
    for v in range(2):
        rec, rect = ludvig.debug_project(sub, wl.cams.params[v], wl.cams.width, wl.cams.height)
        pr = oracle.project(ref_scene, wl.cams.params[v], wl.cams.width, wl.cams.height)
        vis = pr["visible"]
        assert np.array_equal(rect.cpu().numpy(), pr["rect"])
        assert np.array_equal(rec.cpu().numpy()[vis].view(np.uint32), pr["p32"][vis].view(np.uint32))
    o2, b2 = ludvig.uplift(sub, wl.cams.params, wl.cams.width, wl.cams.height, F)
    torch.cuda.synchronize()
    f_ref, b_ref = oracle.uplift(ref_scene, wl.cams, lambda v: wl.features(v))
    pos = b_ref > 0
    e = rel_l2(o2.cpu().numpy(), f_ref, pos)
    print(f"filtered scene: kept {keep} of {sc.n}, uplift rel L2 {e:.2e}")
    assert np.array_equal(b2.cpu().numpy() > 0, pos) and e <= 1e-5


def test_subset_rejects_out_of_range_and_handles_empty():
    sc = _scene_of_size(100)
    bad = torch.tensor([3, 100, 5], dtype=torch.int32, device="cuda")
    with pytest.raises(ludvig.LudvigError, match="ERR_ARG"):
        sc.subset(bad)
    neg = torch.tensor([-1], dtype=torch.int32, device="cuda")
    with pytest.raises(ludvig.LudvigError, match="ERR_ARG"):
        sc.subset(neg)
    empty = sc.subset(torch.zeros((0,), dtype=torch.int32, device="cuda"))
    assert empty.n == 0
    rep = sc.subset(torch.tensor([4, 4, 0], dtype=torch.int32, device="cuda"))
    assert rep.n == 3
