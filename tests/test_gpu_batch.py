"""Packed batches (ludvig_uplift_batch) on one GPU, through the C ABI:

* jobs of four classes (bfloat16 D = 48, bfloat16 D = 3 and float32 D = 1 masks
  on the zero-padded path, float32 D = 40 on the split-bfloat16 path), their features slices of
  shared pools at different view offsets, scenes of uneven size, one job
  without beta: every job equals its own ludvig_uplift run to 1e-5 relative
  L2 (only the order of the atomic sums differs), with groups of one or two
  views (a 1 MiB scratch bound) and with every class in one or two groups;
* the plan reports one class per (dtype, d), the views and the groups;
* with the float32 tensor-core option off, the float32 jobs run as single
  calls and still match;
* a job with an invalid argument fails alone;
* the tuner picks one of its candidate sizes, marks the classes tuned and
  reuses its choice in the next batch;
* a bfloat16 job of the batch meets the bfloat16 bar (1e-2 relative L2)
  against the oracle's float64 uplift of the same bfloat16 values."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_14462_gb300 import inputs, ludvig
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu

W, H, V = 64, 48, 40
SIZES = (9000, 3000, 20000, 500, 6000, 12000)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2410_14462_gb300 import build
    build.build()
    ludvig.load()


@pytest.fixture(scope="module")
def world():
    cams = inputs.cameras_orbit(V, 3.0, W, H, 0.9 * W, hemisphere=True)
    host = [inputs.scene_clusters(n, seed=60 + k, n_clusters=6, sigma=0.2, extent=1.0)
            for k, n in enumerate(SIZES)]
    pools = {48: torch.stack([inputs.feature_field(9, v, 48, H, W, device="cuda") for v in range(V)]
                             ).to(torch.bfloat16).contiguous(),
             3: torch.stack([inputs.feature_field(8, v, 3, H, W, device="cuda") for v in range(V)]
                            ).to(torch.bfloat16).contiguous(),
             40: torch.stack([inputs.feature_field(7, v, 40, H, W, device="cuda") for v in range(V)]
                             ).contiguous(),
             1: inputs.form_pool(1, cams, device="cuda", dtype=torch.float32)}   # float32 sphere masks
    torch.cuda.synchronize()
    return dict(cams=cams, host=host, pools=pools)


@pytest.fixture()
def options():
    """Restores the options a test changes."""
    saved = {o: ludvig.get_option(o) for o in (ludvig.OPT_GROUP_MB, ludvig.OPT_BATCH_TUNE,
                                               ludvig.OPT_F32_TENSOR_CORES)}
    yield
    for o, v in saved.items():
        ludvig.set_option(o, v)


# (scene index, d, first view, views, with beta)
SPECS = [(0, 48, 0, 12, True), (1, 48, 7, 25, True), (2, 48, 30, 10, False), (3, 3, 2, 9, True),
         (4, 3, 11, 17, True), (5, 40, 5, 14, True), (1, 40, 20, 6, True), (3, 48, 1, 3, True),
         (2, 1, 4, 11, True), (5, 1, 25, 7, False)]


def _jobs(world, specs=SPECS):
    scenes = [ludvig.Scene.from_inputs(world["host"][k]) for k, *_ in specs]
    args = []
    for sc, (k, d, v0, nv, with_beta) in zip(scenes, specs):
        out = torch.full((sc.n, d), float("nan"), device="cuda")
        beta = torch.full((sc.n,), float("nan"), device="cuda") if with_beta else None
        args.append((sc, world["cams"].params[v0:v0 + nv], W, H, world["pools"][d][v0:v0 + nv], out, beta))
    return scenes, args


def _run_batch(args, slots=2):
    """uplift_batch with the beta of beta-less jobs left NULL in the job."""
    import ctypes
    L = ludvig.load()
    arr = (ludvig.UpliftJob * len(args))()
    keep = []
    for k, (sc, cp, w, h, f, out, beta) in enumerate(args):
        cams, nv = ludvig.cameras_struct(cp)
        keep.append(cams)
        arr[k] = ludvig.UpliftJob(sc.handle.value, ctypes.addressof(cams), nv, w, h, f.data_ptr(),
                                  ludvig._dtype_code(f), int(f.shape[-1]), out.data_ptr(),
                                  beta.data_ptr() if beta is not None else None)
    status = (ctypes.c_int32 * len(args))()
    rc = L.ludvig_uplift_batch(arr, len(args), slots, status, None)
    torch.cuda.synchronize()
    return rc, [int(status[k]) for k in range(len(args))]


def _check_alone(args, tol=1e-5):
    for sc, cp, w, h, f, out, beta in args:
        a, b = ludvig.uplift(sc, cp, w, h, f)
        torch.cuda.synchronize()
        e = rel_l2(out.cpu().numpy(), a.cpu().numpy())
        assert e <= tol, (sc.n, f.shape, e)
        if beta is not None:
            assert rel_l2(beta.cpu().numpy(), b.cpu().numpy()) <= tol


@pytest.mark.parametrize("group_mb", [1, 2048])
def test_packed_jobs_equal_their_own_runs(world, options, group_mb):
    ludvig.set_option(ludvig.OPT_BATCH_TUNE, 0)
    ludvig.set_option(ludvig.OPT_GROUP_MB, group_mb)
    scenes, args = _jobs(world)
    rc, status = _run_batch(args)
    assert rc == 0 and status == [0] * len(args)
    plan = ludvig.batch_last_plan()
    print(f"group bound {group_mb} MiB: {plan}")
    packed = {(c["dtype"], c["d"]): c for c in plan if c["groups"] >= 0}
    assert set(packed) == {(ludvig.BF16, 48), (ludvig.BF16, 3), (ludvig.F32, 40), (ludvig.F32, 1)}
    assert plan[-1]["groups"] == -1 and plan[-1]["jobs"] == 0
    views = {(ludvig.BF16, 48): 12 + 25 + 10 + 3, (ludvig.BF16, 3): 9 + 17, (ludvig.F32, 40): 14 + 6,
             (ludvig.F32, 1): 11 + 7}
    for key, c in packed.items():
        assert c["views"] == views[key] and c["group_mb"] == group_mb and not c["tuned"]
        if group_mb == 1:
            assert c["groups"] >= c["views"] // 2          # one or two views per group
        else:
            assert c["groups"] <= 2
    _check_alone(args)
    ludvig.set_option(ludvig.OPT_GROUP_MB, 2048)


def test_float32_jobs_run_as_single_calls_without_tensor_cores(world, options):
    ludvig.set_option(ludvig.OPT_BATCH_TUNE, 0)
    ludvig.set_option(ludvig.OPT_F32_TENSOR_CORES, 0)
    scenes, args = _jobs(world)
    rc, status = _run_batch(args, slots=3)
    assert rc == 0 and status == [0] * len(args)
    plan = ludvig.batch_last_plan()
    assert plan[-1]["jobs"] == 4 and plan[-1]["views"] == 14 + 6 + 11 + 7
    assert {(c["dtype"], c["d"]) for c in plan if c["groups"] >= 0} == {(ludvig.BF16, 48), (ludvig.BF16, 3)}
    _check_alone(args)


def test_a_job_with_invalid_arguments_fails_alone(world, options):
    ludvig.set_option(ludvig.OPT_BATCH_TUNE, 0)
    scenes, args = _jobs(world, SPECS[:3])
    sc, cp, w, h, f, out, beta = args[1]
    args[1] = (sc, cp, 0, h, f, out, beta)                  # width 0
    rc, status = _run_batch(args)
    assert rc == 1 and status == [0, 1, 0]
    _check_alone([args[0], args[2]])


def test_tuner_picks_a_candidate_and_reuses_it(world, options):
    ludvig.set_option(ludvig.OPT_BATCH_TUNE, 1)
    ludvig.batch_forget_tuning()
    scenes, args = _jobs(world)
    rc, status = _run_batch(args)
    assert rc == 0 and status == [0] * len(args)
    first = [c for c in ludvig.batch_last_plan() if c["groups"] >= 0]
    print(f"tuned: {first}")
    assert all(c["tuned"] == 1 and c["group_mb"] in (256, 512, 1024, 2048) for c in first)
    _check_alone(args)
    scenes2, args2 = _jobs(world)
    rc, _ = _run_batch(args2)
    assert rc == 0
    again = [c for c in ludvig.batch_last_plan() if c["groups"] >= 0]
    assert {(c["dtype"], c["d"]): c["group_mb"] for c in again} == {(c["dtype"], c["d"]): c["group_mb"] for c in first}


def test_bf16_job_meets_the_bf16_bar_against_the_fp64_oracle(world, options):
    ludvig.set_option(ludvig.OPT_BATCH_TUNE, 0)
    scenes, args = _jobs(world)
    rc, _ = _run_batch(args)
    assert rc == 0
    k = 1                                                     # scene 1 (3000 Gaussians), D = 48, views 7-31
    sc, cp, w, h, f, out, beta = args[k]
    idx, d, v0, nv, _ = SPECS[k]
    cams = inputs.Cameras(world["cams"].params[v0:v0 + nv], W, H)
    X = f.float().cpu().numpy()
    f_ref, b_ref = oracle.uplift(world["host"][idx], cams, lambda v: X[v])
    pos = b_ref > 0
    e = rel_l2(out.cpu().numpy(), f_ref, pos)
    print(f"bf16 job of the batch vs float64 oracle: rel L2 {e:.2e}")
    assert np.array_equal(beta.cpu().numpy() > 0, pos)
    assert e <= 1e-2
