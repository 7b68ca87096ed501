"""GPU parity of the last "next" row through the C ABI:

* ludvig_relevancy (appendix, relevancy scores) against the oracle within
  1e-5 absolute (r lies in [0, 1]; float32 dots of unit vectors, T = 10), for
  1, 21 and 40 queries with 4 canonical phrases, channel counts that are not a
  multiple of the warp, zero feature rows and a row count that is not a
  multiple of the block's rows;
* the GaussianEditor count normaliser (LUDVIG_OPT_COUNT_NORMALISE): the counts
  are bit-exact (the same w > 0 decisions as the contributor counts) and the
  features within the float32 bar (1e-5 relative L2; bfloat16 features 1e-2)
  on the tensor-core and CUDA-core paths."""
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


@pytest.mark.parametrize("n,d,nq", [(5003, 512, 1), (4000, 512, 21), (777, 48, 40), (100, 1024, 20), (1500, 200, 10)])
def test_relevancy_matches_oracle(n, d, nq):
    rng = np.random.default_rng(n + d + nq)
    f = rng.normal(size=(n, d)).astype(np.float32)
    pq = rng.normal(size=(nq, d)).astype(np.float32)
    pc = rng.normal(size=(4, d)).astype(np.float32)
    # make some features close to a query so that scores spread over [0, 1]
    f[1::5] = pq[rng.integers(0, nq, size=f[1::5].shape[0])] + 0.3 * f[1::5]
    f[::97] = 0.0
    r = ludvig.relevancy(torch.from_numpy(f).cuda(), torch.from_numpy(pq).cuda(), torch.from_numpy(pc).cuda(), 10.0)
    got = r.cpu().numpy()
    ref = oracle.relevancy(f, pq, pc, 10.0)
    err = np.abs(got - ref).max()
    print(f"relevancy n={n} d={d} q={nq}: max abs err {err:.2e}, range {ref.min():.3f}..{ref.max():.3f}")
    assert err <= 1e-5
    assert np.all(got[::97] == 0.5)


@pytest.mark.parametrize("d,tc,dtype,gate", [(48, True, torch.float32, 1e-5), (48, False, torch.float32, 1e-5),
                                             (3, True, torch.float32, 1e-5), (40, True, torch.bfloat16, 1e-2)])
def test_count_normalised_uplift(d, tc, dtype, gate):
    wl = inputs.small_field_workload(n=20_000, views=3, d=d, width=100, height=75)
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = device_features(wl, range(3), dtype=dtype)
    old = (ludvig.get_option(ludvig.OPT_F32_TENSOR_CORES), ludvig.get_option(ludvig.OPT_COUNT_NORMALISE))
    ludvig.set_option(ludvig.OPT_F32_TENSOR_CORES, int(tc))
    ludvig.set_option(ludvig.OPT_COUNT_NORMALISE, 1)
    try:
        out, cnt = ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, F)
        torch.cuda.synchronize()
    finally:
        ludvig.set_option(ludvig.OPT_F32_TENSOR_CORES, old[0])
        ludvig.set_option(ludvig.OPT_COUNT_NORMALISE, old[1])
    Fh = F.float().cpu().numpy()
    f_ref, c_ref = oracle.uplift(wl.scene, wl.cams, lambda v: Fh[v], count_normalise=True)
    assert np.array_equal(cnt.cpu().numpy(), c_ref.astype(np.float32)), "counts differ"
    pos = c_ref > 0
    e = rel_l2(out.cpu().numpy(), f_ref, pos)
    print(f"count-normalised uplift d={d} tc={tc} {dtype}: rel L2 {e:.2e}")
    assert e <= gate
