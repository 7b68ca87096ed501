"""Serving and batched forms on one GPU, through the C ABI:

* every request of a concurrent mix (requests on two resident scenes arriving
  together, with and without diffusion, D = 1 masks and two feature widths,
  bfloat16 and float32 pools) gives the same result as when it runs alone: uplift within
  1e-5 relative L2 (only the order of the atomic sums differs), diffused vector
  within 1e-5;
* a request whose outputs exceed the memory budget is rejected and the others
  are served;
* the batched runner finishes jobs of uneven size and each matches its own
  uplift run alone."""
import numpy as np
import pytest
import torch

from paper_2410_14462_gb300 import inputs, ludvig, serve
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2410_14462_gb300 import build
    build.build()
    ludvig.load()


@pytest.fixture(scope="module")
def world():
    W, H, V = 100, 75, 20
    cams = inputs.cameras_orbit(V, 3.0, W, H, 0.9 * W, hemisphere=True)
    host = [inputs.scene_clusters(n, seed=s, n_clusters=8, sigma=0.25, extent=1.0)
            for n, s in ((20_000, 40), (12_000, 41))]
    scenes = [ludvig.Scene.from_inputs(h) for h in host]
    pools = {1: inputs.form_pool(1, cams, device="cuda", dtype=torch.float32)}   # sphere masks
    for d, dt in ((8, torch.float32), (48, torch.bfloat16)):
        pools[d] = torch.stack([inputs.feature_field(7, v, d, H, W, device="cuda") for v in range(V)]
                               ).to(dt).contiguous()
    graphs = []
    for sc in scenes:
        f, _ = ludvig.uplift(sc, cams.params[:4], W, H, pools[48][:4].contiguous())
        graphs.append(ludvig.Graph(sc, 8, f, spatial_h=0.01))
    torch.cuda.synchronize()
    return dict(W=W, H=H, V=V, cams=cams, host=host, scenes=scenes, pools=pools, graphs=graphs)


def _server(w, budget=1 << 34, slots=2):
    return serve.Server(w["scenes"], w["graphs"], w["pools"], w["cams"].params, w["W"], w["H"], budget, slots)


def test_results_same_alone_and_in_the_mix(world):
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(12):
        views = int(rng.integers(2, 9))
        reqs.append(serve.Request(i, 0.0, i % 2, [8, 48, 1][(i // 2) % 3], int(rng.integers(0, world["V"] - views)),
                                  views, diffuse_iters=[0, 15][i % 3 == 0 or i % 4 == 0], keep_output=True))
    srv = _server(world, slots=3)
    mixed = srv.run(reqs)
    srv.close()
    assert all(r.ok for r in mixed), [r.error for r in mixed if not r.ok]
    single = _server(world, slots=1)
    for req, rm in zip(reqs, mixed):
        alone = single.run([serve.Request(req.rid, 0.0, req.scene, req.d, req.v0, req.views,
                                          req.diffuse_iters, True)])[0]
        assert alone.ok
        e = rel_l2(rm.out.cpu().numpy(), alone.out.cpu().numpy())
        assert e <= 1e-5, (req, e)
        if req.diffuse_iters:
            assert rel_l2(rm.g.cpu().numpy(), alone.g.cpu().numpy()) <= 1e-5
    s = serve.latency_summary(mixed)
    print(f"mix: {s}")
    assert s["served"] == 12 and s["p99_ms"] >= s["p50_ms"] > 0


def test_poisoned_request_leaves_the_others_intact(world):
    """A request whose features are all NaN (its own pool) shares the GPU with
    two clean requests on the same scene: its output is not finite, theirs
    equal their runs alone (outputs are per-request buffers, and no kernel's
    control flow depends on feature values)."""
    V, H, W = world["V"], world["H"], world["W"]
    pools = dict(world["pools"])
    pools[16] = torch.full((V, H, W, 16), float("nan"), dtype=torch.float32, device="cuda")
    srv = serve.Server(world["scenes"], world["graphs"], pools, world["cams"].params, W, H, 1 << 34, 3)
    reqs = [serve.Request(0, 0.0, 0, 8, 0, 5, keep_output=True), serve.Request(1, 0.0, 0, 16, 2, 5, keep_output=True),
            serve.Request(2, 0.0, 0, 48, 4, 5, keep_output=True)]
    res = srv.run(reqs)
    srv.close()
    assert res[0].ok and res[2].ok
    assert (not res[1].ok) or not bool(torch.isfinite(res[1].out).all())
    single = _server(world, slots=1)
    for k in (0, 2):
        q = reqs[k]
        alone = single.run([serve.Request(q.rid, 0.0, q.scene, q.d, q.v0, q.views, 0, True)])[0]
        assert rel_l2(res[k].out.cpu().numpy(), alone.out.cpu().numpy()) <= 1e-5


def test_admission_rejects_requests_over_budget(world):
    """The budget covers the server's replicas and the live workspaces besides
    the outputs: with room for the workspaces (grown first by two requests of the
    small requests' shape), one small output and 2 MB, the large request
    on scene 0 is rejected and the small ones on scene 1 are served."""
    srv = _server(world, 1 << 40, slots=2)
    res_bytes = srv.resident_bytes()
    assert res_bytes >= serve.SCENE_BYTES_PER_GAUSSIAN * sum(sc.n for sc in world["scenes"])   # one replica each
    assert res_bytes >= sum(sc.workspace_bytes() for sc in world["scenes"]) > 0
    srv.close()
    srv = _server(world, 1 << 40, slots=1)
    # the small requests' shape once, so that the replica's workspace already
    # holds what they need (a workspace grows to the largest request it served)
    assert all(r.ok for r in srv.run([serve.Request(0, 0.0, 1, 8, 0, 4), serve.Request(1, 0.0, 1, 8, 4, 4)]))
    srv.budget = srv.resident_bytes() + serve.request_bytes(world["scenes"][1].n, 8) + (2 << 20)
    assert serve.request_bytes(world["scenes"][0].n, 48) > serve.request_bytes(world["scenes"][1].n, 8) + (2 << 20)
    reqs = [serve.Request(0, 0.0, 0, 48, 0, 4), serve.Request(1, 0.0, 1, 8, 0, 4),
            serve.Request(2, 0.01, 1, 8, 4, 4)]
    res = srv.run(reqs)
    assert not res[0].ok and "budget" in res[0].error
    assert res[1].ok and res[2].ok


def test_batched_jobs_match_their_own_runs(world):
    scenes = [world["scenes"][j % 2] if j < 2 else ludvig.Scene.from_inputs(world["host"][j % 2]) for j in range(6)]
    jobs = [serve.Job(j, scenes[j], [8, 48][j % 2], j, 3 + j) for j in range(6)]
    res = serve.run_batch(jobs, world["pools"], world["cams"].params, world["W"], world["H"], slots=3,
                          keep_outputs=True)
    assert not res["errors"] and len(res["outputs"]) == 6
    for j in jobs:
        a, b = ludvig.uplift(j.scene, world["cams"].params[j.v0:j.v0 + j.views], world["W"], world["H"],
                             world["pools"][j.d][j.v0:j.v0 + j.views])
        out, beta = res["outputs"][j.jid]
        assert rel_l2(out.cpu().numpy(), a.cpu().numpy()) <= 1e-5
        assert rel_l2(beta.cpu().numpy(), b.cpu().numpy()) <= 1e-5
    for sc in scenes[2:]:
        sc.close()
    # the slots' pooled workspaces hold device memory until released
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ludvig.batch_release_workspaces()
    assert torch.cuda.mem_get_info()[0] > free0
    ludvig.batch_release_workspaces()   # an empty pool is fine


def test_uplift_batch_abi_errors_and_job_status(world):
    """Argument errors come before any work (a scene in two jobs, slots out of
    range); a job that fails its own checks reports its status while the
    other jobs of the batch still run to the right result."""
    W, H, cams, pools = world["W"], world["H"], world["cams"].params, world["pools"]
    s0, s1 = world["scenes"]
    job = lambda sc, d, views: (sc, cams[:views], W, H, pools[d][:views], None, None)
    with pytest.raises(ludvig.LudvigError, match="share a scene"):
        ludvig.uplift_batch([job(s0, 8, 2), job(s0, 48, 2)])
    with pytest.raises(ludvig.LudvigError, match="slots"):
        ludvig.uplift_batch([job(s0, 8, 2)], slots=0)
    with pytest.raises(ludvig.LudvigError, match="slots"):
        ludvig.uplift_batch([job(s0, 8, 2)], slots=ludvig.MAX_BATCH_SLOTS + 1)
    bad = np.array(cams[:2], copy=True)
    bad[:, 12] = 0.0                                    # fx = 0: the job's own argument check fails
    bad_job = (s1, bad, W, H, pools[8][:2], None, None)
    res, status = ludvig.uplift_batch([job(s0, 48, 3), bad_job], slots=2, raise_on_error=False)
    assert status[0] == 0 and status[1] == ludvig.ERR_ARG
    with pytest.raises(ludvig.LudvigError, match="job 1"):
        ludvig.uplift_batch([job(s0, 48, 3), bad_job], slots=2)
    a, b = ludvig.uplift(s0, cams[:3], W, H, pools[48][:3])
    assert rel_l2(res[0][0].cpu().numpy(), a.cpu().numpy()) <= 1e-5
    assert ludvig.uplift_batch([], slots=3) == ([], [])
