"""GPU parity of the tensor-core (tcgen05) aggregation used for bfloat16
features (the precision form of Sec. 3.2 Eq. 3), through the C ABI.

* the product primitive itself, W_tile (128 x 256) . F_tile (256 x d), against
  a float32 matmul of the same bfloat16 values (products of bfloat16 values are
  exact in float32, so only the summation order differs: 1e-5 relative);
* structured operands that expose a wrong shared-memory layout;
* the full uplift against the float64 oracle: within 1e-2 relative L2 of the
  oracle on the original float32 features (weights rounded to bfloat16 for the
  product, beta summing the same rounded weights), and a constant map
  reproduced to float32 rounding (each f_i stays a convex combination)."""
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


@pytest.mark.parametrize("d", [64, 128, 320, 512])
def test_tile_product_matches_matmul(d):
    g = torch.Generator(device="cpu").manual_seed(d)
    a = torch.randn((128, 256), generator=g).to(torch.bfloat16).cuda()
    f = torch.randn((16, 16, d), generator=g).to(torch.bfloat16).cuda()
    out = ludvig.debug_mma_bf16(a, f)
    ref = a.float() @ f.reshape(256, d).float()
    torch.cuda.synchronize()
    e = (out - ref).norm() / ref.norm()
    print(f"d={d}: rel err {e.item():.2e}")
    assert e.item() < 1e-5


def test_tile_product_structure():
    d = 128
    # a selects pixel p = (3 * r) % 256 for row r: out[r] must equal f[p]
    a = torch.zeros((128, 256), dtype=torch.bfloat16)
    sel = [(3 * r) % 256 for r in range(128)]
    for r, p in enumerate(sel):
        a[r, p] = 1.0
    f = torch.arange(256 * d, dtype=torch.float32).reshape(16, 16, d) % 251
    out = ludvig.debug_mma_bf16(a.cuda(), f.to(torch.bfloat16).cuda()).cpu()
    fr = f.reshape(256, d)
    bad = [r for r in range(128) if not torch.equal(out[r], fr[sel[r]])]
    assert not bad, f"rows {bad[:8]} wrong; row 0 got {out[bad[0], :8].tolist()} want {fr[sel[bad[0]], :8].tolist()}"


def _bf16_uplift(wl, views):
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = device_features(wl, views, torch.bfloat16)
    out, beta = ludvig.uplift(sc, wl.cams.params[views], wl.cams.width, wl.cams.height, F)
    torch.cuda.synchronize()
    return out.cpu().numpy(), beta.cpu().numpy(), F


@pytest.mark.parametrize("d", [64, 192, 512])
def test_tc_uplift_matches_oracle(d):
    wl = inputs.small_field_workload(n=20_000, views=3, d=d, width=100, height=75)
    out, beta, F = _bf16_uplift(wl, [0, 1, 2])
    f32, b32 = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v))
    Fh = F.float().cpu().numpy()
    fbf, bbf = oracle.uplift(wl.scene, wl.cams, lambda v: Fh[v])
    pos = b32 > 0
    assert np.array_equal(beta > 0, pos)
    e32 = rel_l2(out, f32, pos)
    ebf = rel_l2(out, fbf, pos)
    eb = rel_l2(beta, b32)
    print(f"d={d}: bf16 tensor-core uplift rel L2 vs float64 oracle: {e32:.2e} (float32 features), "
          f"{ebf:.2e} (same bf16 features); beta {eb:.2e}")
    assert e32 <= 1e-2 and ebf <= 1e-2 and eb <= 1e-2


def test_tc_constant_map_is_exact():
    wl = inputs.small_field_workload(n=20_000, views=3, d=128, width=100, height=75)
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = torch.full((3, 75, 100, 128), 0.5, dtype=torch.bfloat16, device="cuda")
    F[..., 1::2] = -2.0
    out, beta = ludvig.uplift(sc, wl.cams.params, 100, 75, F)
    torch.cuda.synchronize()
    out, beta = out.cpu().numpy(), beta.cpu().numpy()
    pos = beta > 0
    assert pos.sum() > 5000
    np.testing.assert_allclose(out[pos, 0::2], 0.5, rtol=2e-6)
    np.testing.assert_allclose(out[pos, 1::2], -2.0, rtol=2e-6)


def test_tc_dense_stack_many_flushes():
    """Long lists of weak splats: many 128-row W tiles per item."""
    rng = np.random.default_rng(0)
    n = 3000
    sc_in = inputs.Scene((rng.normal(size=(n, 3)) * 0.05).astype(np.float32), np.full((n, 3), 0.2, np.float32),
                         rng.normal(size=(n, 4)).astype(np.float32), np.full(n, 0.02, np.float32))
    cams = inputs.cameras_orbit(2, 3.0, 96, 64, 100.0, hemisphere=True)
    Ff = torch.rand((2, 64, 96, 64), device="cuda")
    F = Ff.to(torch.bfloat16)
    sc = ludvig.Scene.from_inputs(sc_in)
    out, beta = ludvig.uplift(sc, cams.params, 96, 64, F)
    Fh = F.float().cpu().numpy()
    f_ref, b_ref = oracle.uplift(sc_in, cams, lambda v: Fh[v])
    torch.cuda.synchronize()
    pos = b_ref > 0
    e = rel_l2(out.cpu().numpy(), f_ref, pos)
    print(f"dense stack: rel L2 {e:.2e}")
    assert e <= 1e-2
