"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point that include/ludvig.h declares, and rejects bad arguments
synchronously (no CUDA call is made on those paths)."""
import ctypes
import os
import re

import pytest

from paper_2410_14462_gb300 import build, ludvig

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ludvig.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ludvig_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ludvig.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
    # and the binding covers the same set
    assert set(names) == set(ludvig.SIGNATURES)


def test_abi_version(lib):
    assert lib.ludvig_abi_version() == 11


def test_argument_errors_are_synchronous(lib):
    h = ctypes.c_void_p()
    assert lib.ludvig_scene_create(None, None, None, None, 5, None, None, ctypes.byref(h)) == 1
    assert b"NULL" in lib.ludvig_last_error()
    assert lib.ludvig_scene_create(None, None, None, None, -1, None, None, ctypes.byref(h)) == 1
    assert lib.ludvig_sync(None) == 1
    assert lib.ludvig_debug_scene_timeout(None, 10, None) == 1
    assert lib.ludvig_uplift(None, None, 1, 64, 64, None, 0, 4, None, None, None) == 1
    assert lib.ludvig_knn(None, 4, None, None) == 1
    assert lib.ludvig_render(None, None, 1, 64, 64, None, 4, None, None) == 1
    assert lib.ludvig_beta_select(None, None, 1, None, None) == 1
    h2 = ctypes.c_void_p()
    assert lib.ludvig_scene_subset(None, None, 1, None, ctypes.byref(h2)) == 1
    assert lib.ludvig_diffuse(None, None, 1, 1, None, None) == 1
    assert lib.ludvig_uplift_finalize(-1, 4, None, None, None, None, None) == 1
    assert lib.ludvig_scene_size(None) == -1
    assert lib.ludvig_graph_nnz(None) == -1
    assert lib.ludvig_scene_workspace_bytes(None) == -1
    assert lib.ludvig_graph_workspace_bytes(None) == -1
    assert lib.ludvig_scene_destroy(None) == 0


def test_batch_argument_errors_are_synchronous(lib):
    """ludvig_uplift_batch checks its arguments before touching a scene or the
    GPU: negative counts, NULL jobs, slots out of range, a NULL scene and a
    scene shared by two jobs (the handles below are never dereferenced)."""
    Job = ludvig.UpliftJob
    status = (ctypes.c_int32 * 2)()
    assert lib.ludvig_uplift_batch(None, 0, 4, None, None) == 0        # nothing to do
    assert lib.ludvig_uplift_batch(None, -1, 4, None, None) == 1
    assert lib.ludvig_uplift_batch(None, 2, 4, status, None) == 1
    jobs = (Job * 2)()
    jobs[0].scene = jobs[1].scene = 0x1000                             # same (fake) handle
    for slots in (0, ludvig.MAX_BATCH_SLOTS + 1):
        assert lib.ludvig_uplift_batch(jobs, 2, slots, status, None) == 1
        assert b"slots" in lib.ludvig_last_error()
    assert lib.ludvig_uplift_batch(jobs, 2, 2, status, None) == 1
    assert b"share a scene" in lib.ludvig_last_error()
    jobs[1].scene = None
    assert lib.ludvig_uplift_batch(jobs, 2, 2, status, None) == 1
    assert b"job 1: scene is NULL" in lib.ludvig_last_error()
    assert ctypes.sizeof(Job) == 64                                    # matches ludvig_uplift_job


def test_diffusion_wrappers_check_shapes_before_launch(lib):
    """Graph.diffuse and Graph.diffuse_noalloc reject an x0 whose first
    dimension is not the graph's n, an x0 of rank 3 and an out of another
    shape, before any library call (the handle here is never used)."""
    import torch
    g = ludvig.Graph.__new__(ludvig.Graph)
    g.n = 10
    g._h = None
    ok = torch.zeros(10, 3)
    for x0, out in ((torch.zeros(9), None), (torch.zeros(10, 2, 2), None), (ok, torch.zeros(10, 2)),
                    (torch.zeros(10), torch.zeros(10, 1))):
        with pytest.raises(ludvig.LudvigError, match="x0|out"):
            g.diffuse(x0, 3, out=out)
        with pytest.raises(ludvig.LudvigError, match="x0|out"):
            g.diffuse_noalloc(x0, 3, out if out is not None else torch.zeros_like(x0))
