"""GPU parity of the rendering operator F_hat = W f (Sec. 3.2, Eq. 4) against the
CPU oracle, through the C ABI (ludvig_render).

Bars: relative L2 <= 1e-5 against the float64 oracle over every element, for
the tensor-core kernel (split-bfloat16 operands: each product keeps 16
significant bits of w and of f, relative error below 3 * 2^-18 per term) and
for the CUDA-core kernel (float32); pixels without a contributor are exactly
zero on both paths.  Cases span several tiles with ragged image edges, channel
blocks with a ragged tail (d = 136), every CUDA-core channel width, and the
degenerate cases (no views, an empty scene, every Gaussian behind the camera,
images smaller than a tile)."""
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


def _render(wl, f, views, tensor_cores=True):
    sc = ludvig.Scene.from_inputs(wl.scene)
    ft = torch.from_numpy(f).cuda()
    old = ludvig.get_option(ludvig.OPT_F32_TENSOR_CORES)
    ludvig.set_option(ludvig.OPT_F32_TENSOR_CORES, int(tensor_cores))
    try:
        out = torch.full((len(views), wl.cams.height, wl.cams.width, f.shape[1]), float("nan"), device="cuda")
        ludvig.render(sc, wl.cams.params[views], wl.cams.width, wl.cams.height, ft, out=out)
        torch.cuda.synchronize()
    finally:
        ludvig.set_option(ludvig.OPT_F32_TENSOR_CORES, old)
    return out.cpu().numpy()


@pytest.mark.parametrize("d,tc", [(48, True), (48, False), (136, True), (3, False), (13, False), (32, True),
                                  (512, True)])
def test_render_matches_oracle(d, tc):
    wl = inputs.small_field_workload(n=20_000, views=3, d=d, width=100, height=75)
    views = [0, 1, 2] if d < 512 else [1]
    f = inputs.gaussian_features(wl.scene.n, d, seed=d)
    got = _render(wl, f, views, tensor_cores=tc)
    ref = oracle.render(wl.scene, wl.cams, f, views=views)
    assert np.isfinite(got).all(), "every output element is written"
    e = rel_l2(got, ref)
    zero = np.abs(ref).max(axis=-1) == 0
    print(f"render d={d} {'tensor cores' if tc else 'CUDA cores'}: rel L2 {e:.2e}, "
          f"max abs {np.abs(got - ref).max():.2e}, {zero.sum()} empty pixels")
    assert e <= 1e-5
    assert (got[zero] == 0).all()
    assert zero.any() and (~zero).sum() > 1000


def test_render_ones_is_one_minus_transmittance():
    """f = 1 renders 1 - T_final (Eq. 1 telescopes); T_final from the GPU's
    own compositing walk, so the two kernels see the same weights."""
    wl = inputs.small_field_workload(n=20_000, views=2, d=32, width=100, height=75)
    sc = ludvig.Scene.from_inputs(wl.scene)
    for tc, d in ((True, 32), (False, 4)):
        got = _render(wl, np.ones((wl.scene.n, d), np.float32), [0, 1], tensor_cores=tc)
        for v in range(2):
            t, _ = ludvig.debug_transmittance(sc, wl.cams.params[v], wl.cams.width, wl.cams.height)
            err = np.abs(got[v] - (1.0 - t.cpu().numpy())[..., None]).max()
            print(f"ones d={d} tc={tc} view {v}: max |F_hat - (1 - T)| = {err:.2e}")
            assert err < 2e-5


def test_adjoint_with_gpu_uplift_numerator():
    """<W f, F> = <f, W^T F> with both sides from the GPU (render, and the
    uplift's accumulation), float64 dot products."""
    wl = inputs.small_field_workload(n=20_000, views=3, d=64, width=100, height=75)
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = device_features(wl, range(3))
    num = torch.zeros((sc.n, 64), device="cuda")
    den = torch.zeros((sc.n,), device="cuda")
    ludvig.uplift_accumulate(sc, wl.cams.params, wl.cams.width, wl.cams.height, F, num, den)
    f = inputs.gaussian_features(sc.n, 64, seed=9)
    Fh = _render(wl, f, [0, 1, 2])
    lhs = float(np.sum(Fh.astype(np.float64) * F.cpu().numpy().astype(np.float64)))
    rhs = float(np.sum(f.astype(np.float64) * num.cpu().numpy().astype(np.float64)))
    print(f"adjoint: <Wf,F> = {lhs:.8e}, <f,W^T F> = {rhs:.8e}")
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.sum(Fh.astype(np.float64) ** 2) * np.sum(F.cpu().numpy() ** 2.0))


def test_render_is_deterministic():
    wl = inputs.small_field_workload(n=20_000, views=2, d=64, width=100, height=75)
    f = inputs.gaussian_features(wl.scene.n, 64, seed=4)
    a = _render(wl, f, [0, 1])
    b = _render(wl, f, [0, 1])
    assert np.array_equal(a, b)


def test_render_edge_cases():
    wl = inputs.tiny_mask_workload()
    W, H = wl.cams.width, wl.cams.height
    empty = inputs.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32),
                         np.zeros((0, 4), np.float32), np.zeros((0,), np.float32))
    sc0 = ludvig.Scene.from_inputs(empty)
    out = torch.full((2, H, W, 40), float("nan"), device="cuda")
    ludvig.render(sc0, wl.cams.params[:2], W, H, torch.zeros((0, 40), device="cuda"), out=out)
    torch.cuda.synchronize()
    assert (out == 0).all()
    sc = ludvig.Scene.from_inputs(wl.scene)
    f = torch.from_numpy(inputs.gaussian_features(sc.n, 40, seed=1)).cuda()
    out = ludvig.render(sc, wl.cams.params[:0], W, H, f)
    assert out.shape == (0, H, W, 40)
    # every Gaussian behind the camera: all zero on both paths
    cam = wl.cams.params[:1].copy()
    cam[0, 9:12] = [0, 0, -50.0]
    for d in (40, 5):
        o = torch.full((1, H, W, d), float("nan"), device="cuda")
        ludvig.render(sc, cam, W, H, f[:, :d].contiguous(), out=o)
        torch.cuda.synchronize()
        assert (o == 0).all()
    # a one-pixel image and one narrower than a tile
    for (w, h) in [(1, 1), (5, 37)]:
        cams = inputs.cameras_orbit(2, 3.0, w, h, 120.0, hemisphere=False)
        small = inputs.Workload("small", wl.scene, cams, 40, 0, "field")
        fn = f.cpu().numpy()
        got = _render(small, fn, [0, 1])
        ref = oracle.render(wl.scene, cams, fn)
        assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("d,tc", [(40, True), (5, False)])
def test_render_spans_view_chunks(d, tc):
    """20 views run as two launches (16 + 4 views); each view's map must land
    at its own offset of the output."""
    wl = inputs.small_field_workload(n=8000, views=20, d=d, width=45, height=37)
    f = inputs.gaussian_features(wl.scene.n, d, seed=30 + d)
    views = list(range(20))
    got = _render(wl, f, views, tensor_cores=tc)
    ref = oracle.render(wl.scene, wl.cams, f, views=views)
    assert np.isfinite(got).all()
    for v in (0, 15, 16, 19):
        assert rel_l2(got[v], ref[v]) <= 1e-5, v
    assert rel_l2(got, ref) <= 1e-5
