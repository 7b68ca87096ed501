"""GPU parity of the FP8-E4M3 feature storage through the C ABI: the per-view
scales and every code are bit-exact against the oracle's quantiser (float32
and bfloat16 inputs, an all-zero view, totals that are not a multiple of 4);
the uplift of the codes meets the bfloat16 bar (1e-2 relative L2) against
the oracle's float64 uplift of the decoded values, on the tensor-core path
(D = 48) and the padded one (D = 3); and the codes decoded inside the
aggregation give the bfloat16 uplift of the same decoded values."""
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


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(5, 13, 17, 3), (3, 48, 64, 64)])
def test_quantize_bitexact(dtype, shape):
    rng = np.random.default_rng(shape[-1])
    x = rng.normal(size=shape).astype(np.float32) * np.array([1e-3, 1.0, 40.0, 0.5, 2.0][: shape[0]],
                                                             np.float32).reshape(-1, 1, 1, 1)
    x[1] = 0.0                                          # an all-zero view: scale 1, codes 0
    xt = torch.from_numpy(x).to(dtype).cuda()
    q, s = ludvig.fp8_quantize(xt)
    torch.cuda.synchronize()
    qr, sr = oracle.fp8_quantize(xt.float().cpu().numpy())
    assert np.array_equal(s.cpu().numpy(), sr)
    assert np.array_equal(q.cpu().numpy(), qr)
    assert s[1].item() == 1.0 and (q[1] == 0).all()


@pytest.mark.parametrize("d", [48, 3])
def test_uplift_fp8_matches_oracle(d):
    wl = inputs.small_field_workload(n=8000, views=3, d=d, width=61, height=45)
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = torch.stack([wl.features(v, device="cuda") for v in range(3)]).contiguous()
    q, s = ludvig.fp8_quantize(F)
    out, beta = ludvig.uplift_fp8(sc, wl.cams.params, wl.cams.width, wl.cams.height, q, s)
    o32, b32 = ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, F)
    torch.cuda.synchronize()
    X = oracle.fp8_dequantize(q.cpu().numpy(), s.cpu().numpy())
    f_ref, b_ref = oracle.uplift(wl.scene, wl.cams, lambda v: X[v])
    pos = b_ref > 0
    assert np.array_equal(beta.cpu().numpy() > 0, pos)
    e = rel_l2(out.cpu().numpy(), f_ref, pos)
    e32 = rel_l2(out.cpu().numpy(), o32.cpu().numpy(), pos)
    print(f"fp8 d={d}: rel L2 vs oracle on the decoded values {e:.2e}; vs the float32 path on the field {e32:.2e}")
    assert e <= 1e-2
    assert rel_l2(beta.cpu().numpy(), b_ref) <= 1e-2


def test_fp8_arguments():
    sc = ludvig.Scene.from_inputs(inputs.scene_uniform(100, seed=0))
    cams = inputs.cameras_orbit(2, 3.0, 16, 16, 20.0, hemisphere=False)
    q = torch.zeros((2 * 16 * 16 * 4 + 1,), dtype=torch.uint8, device="cuda")
    s = torch.ones((2,), dtype=torch.float32, device="cuda")
    with pytest.raises(ludvig.LudvigError, match="aligned"):
        ludvig.uplift_fp8(sc, cams.params, 16, 16, q[1:].view(2, 16, 16, 4), s)
    out, beta = ludvig.uplift_fp8(sc, cams.params, 16, 16, q[:-1].view(2, 16, 16, 4), s)   # all-zero codes
    torch.cuda.synchronize()
    assert (out == 0).all()
    q0, s0 = ludvig.fp8_quantize(torch.zeros((0, 4), device="cuda"))
    assert q0.numel() == 0 and s0.numel() == 0


@pytest.mark.parametrize("d,views,group_mb", [(48, 3, 2048), (64, 20, 1), (40, 3, 2048), (3, 7, 1), (512, 2, 2048)])
def test_uplift_fp8_equals_bf16_uplift_of_the_decoded_values(d, views, group_mb):
    """The aggregation decodes the codes itself when d % 16 == 0 (d = 48, 64,
    512; with a 1 MiB group bound every view is a group of its own, so the
    scales are indexed by the views' coordinates across groups); d = 40 and
    d = 3 take the decode pass (d = 3 with one-view groups: a view holds an
    odd number of codes, so most groups' codes are not 4-byte aligned).  Either way the result is the
    bfloat16 uplift of x = decode(q) s_v rounded to bfloat16, here decoded by
    torch's float8_e4m3fn (float32 product, then bfloat16), to float32
    rounding (only the order of the atomic sums differs)."""
    wl = inputs.small_field_workload(n=8000, views=views, d=d, width=61, height=45)
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = torch.stack([wl.features(v, device="cuda") for v in range(views)]).contiguous()
    q, s = ludvig.fp8_quantize(F)
    saved = ludvig.get_option(ludvig.OPT_GROUP_MB)
    ludvig.set_option(ludvig.OPT_GROUP_MB, group_mb)
    try:
        out, beta = ludvig.uplift_fp8(sc, wl.cams.params, wl.cams.width, wl.cams.height, q, s)
    finally:
        ludvig.set_option(ludvig.OPT_GROUP_MB, saved)
    X = (q.view(torch.float8_e4m3fn).float() * s.view(-1, 1, 1, 1)).to(torch.bfloat16).contiguous()
    ob, bb = ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, X)
    torch.cuda.synchronize()
    e = rel_l2(out.cpu().numpy(), ob.cpu().numpy())
    print(f"fp8 d={d}, {views} views: rel L2 vs the bfloat16 uplift of the decoded values {e:.2e}")
    assert e <= 1e-6
    assert rel_l2(beta.cpu().numpy(), bb.cpu().numpy()) <= 1e-6
