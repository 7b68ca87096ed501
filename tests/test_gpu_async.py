"""The asynchronous uplift contract through the C ABI (the conventions of
include/ludvig.h):

* ludvig_uplift returns without waiting on the host: it returns while a long
  kernel queued ahead of it on the same stream is still running, and the
  result is the oracle's once ludvig_sync has returned;
* ludvig_sync reports the scene's device status word (a bounded wait that
  expires on purpose, without any fault) once, and clears it;
* groups of views that outgrow the workspace sized by an earlier, smaller
  call add nothing on the device and are redone by ludvig_sync: the result
  still matches the float64 oracle (Sec. 3.2, Eq. 3), for the pair buffers and
  for the weight-row chunks."""
import ctypes
import time

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


def _check_oracle(wl, out, views, tol=1e-5):
    f_ref, b_ref = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v), views=views)
    pos = b_ref > 0
    err = rel_l2(out.cpu().numpy(), f_ref, pos)
    print(f"rel L2 vs float64 oracle: {err:.3e}")
    assert err <= tol
    return f_ref, b_ref


def test_uplift_returns_before_the_gpu_finishes():
    wl = inputs.small_field_workload(n=20_000, views=4, d=48, width=100, height=75)
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = device_features(wl, range(4))
    W, H = wl.cams.width, wl.cams.height
    ludvig.uplift(sc, wl.cams.params, W, H, F)          # sizes the workspace
    torch.cuda.synchronize()
    out = torch.full((sc.n, 48), float("nan"), device="cuda")
    beta = torch.empty((sc.n,), device="cuda")
    torch.cuda._sleep(400_000_000)                       # about 0.2 s of SM clock ahead of the uplift
    t0 = time.perf_counter()
    ludvig.uplift(sc, wl.cams.params, W, H, F, out, beta, sync=False)
    dt = time.perf_counter() - t0
    ev = torch.cuda.Event()
    ev.record()
    still_running = not ev.query()
    sc.sync()
    torch.cuda.synchronize()
    print(f"ludvig_uplift returned after {dt * 1e3:.2f} ms; queue still busy: {still_running}")
    assert still_running, "the call waited for the GPU"
    _check_oracle(wl, out, range(4))


def test_sync_reports_the_scene_status_once():
    L = ludvig.load()
    wl = inputs.small_field_workload(n=5000, views=2, d=40, width=61, height=45)
    sc = ludvig.Scene.from_inputs(wl.scene)
    assert L.ludvig_debug_scene_timeout(sc.handle, 2_000_000, None) == 0   # enqueued, not waited for
    rc = L.ludvig_sync(sc.handle)
    assert rc == 4, ludvig.STATUS.get(rc)                                   # LUDVIG_ERR_TIMEOUT
    assert b"expired" in L.ludvig_last_error()
    assert L.ludvig_sync(sc.handle) == 0                                    # reported once
    assert L.ludvig_debug_scene_timeout(None, 1, None) == 1
    assert L.ludvig_debug_scene_timeout(sc.handle, -1, None) == 1
    # the scene and the context keep working
    out, _ = ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, device_features(wl, range(2)))
    torch.cuda.synchronize()
    _check_oracle(wl, out, range(2))


def _dense_scene(n=20_000, seed=11):
    """A thin, dense slab of faint Gaussians: seen from afar it covers few
    tiles; from near, every tile holds hundreds of contributors (many more
    pairs and weight rows than the far view)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.3, 0.3, size=(n, 3)) * np.array([1.0, 1.0, 0.2])
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return inputs.Scene(means.astype(np.float32), np.full((n, 3), 0.03, np.float32), q.astype(np.float32),
                        np.full(n, 0.05, np.float32))


@pytest.mark.parametrize("d", [48, 3])
def test_groups_that_outgrow_the_workspace_are_redone(d):
    scene = _dense_scene()
    far = inputs.cameras_orbit(2, 25.0, 16, 16, 90.0, hemisphere=True)   # one tile
    near = inputs.cameras_orbit(18, 1.6, 96, 80, 90.0, hemisphere=True)
    wl_far = inputs.Workload("dense-far", scene, far, d, 5, "field")
    wl_near = inputs.Workload("dense-near", scene, near, d, 5, "field")
    sc = ludvig.Scene.from_inputs(scene)
    ludvig.uplift(sc, far.params, far.width, far.height, device_features(wl_far, range(far.v)))
    torch.cuda.synchronize()
    L = ludvig.load()
    # the far call sized the workspace; the near views need far more of it
    F = device_features(wl_near, range(near.v))
    probe = ludvig.Scene.from_inputs(scene)   # (its checked runs would grow sc's workspace)
    ranges, _ = ludvig.debug_tile_lists(probe, near.params[0], near.width, near.height)
    r_far, _ = ludvig.debug_tile_lists(probe, far.params[0], far.width, far.height)
    pairs_near = int((ranges[:, 1] - ranges[:, 0]).sum())
    pairs_far = int((r_far[:, 1] - r_far[:, 0]).sum())
    print(f"pairs per view: far {pairs_far}, near {pairs_near}")
    # the near views need several times what the 2 far views did
    assert 16 * pairs_near > 8 * 2 * max(pairs_far, 1)
    out = torch.empty((sc.n, d), device="cuda")
    beta = torch.empty((sc.n,), device="cuda")
    ludvig.uplift(sc, near.params, near.width, near.height, F, out, beta, sync=False)
    assert L.ludvig_sync(sc.handle) == 0
    torch.cuda.synchronize()
    f_ref, b_ref = _check_oracle(wl_near, out, range(near.v))
    assert np.array_equal(beta.cpu().numpy() > 0, b_ref > 0)
    # the workspace has grown: the same call now fits on the device
    out2, _ = ludvig.uplift(sc, near.params, near.width, near.height, F)
    torch.cuda.synchronize()
    assert rel_l2(out2.cpu().numpy(), f_ref, b_ref > 0) <= 1e-5


@pytest.mark.parametrize("d,dtype", [(48, torch.bfloat16), (3, torch.float32), (40, torch.float32)])
def test_many_groups_equal_one_group(d, dtype):
    """With a 1 MiB group bound each of the 12 views is a group of its own
    (12 asynchronous groups on alternating buffer sets); the result equals
    the one-group call's to float32 rounding."""
    wl = inputs.small_field_workload(n=8000, views=12, d=d, width=61, height=45)
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = device_features(wl, range(12), dtype)
    one, b1 = ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, F)
    saved = ludvig.get_option(ludvig.OPT_GROUP_MB)
    ludvig.set_option(ludvig.OPT_GROUP_MB, 1)
    try:
        many, bm = ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, F)
    finally:
        ludvig.set_option(ludvig.OPT_GROUP_MB, saved)
    torch.cuda.synchronize()
    assert rel_l2(many.cpu().numpy(), one.cpu().numpy()) <= 1e-5
    assert rel_l2(bm.cpu().numpy(), b1.cpu().numpy()) <= 1e-5
