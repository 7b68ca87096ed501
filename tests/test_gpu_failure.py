"""Failure detection without a GPU fault: a bounded device wait on an mbarrier
that nothing arrives on expires after its budget, the kernel records
LUDVIG_ERR_TIMEOUT and returns, the host reads that status, and the context
keeps working (a normal uplift afterwards matches the oracle)."""
import ctypes

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


def test_bounded_wait_expires_and_context_survives():
    L = ludvig.load()
    waited = ctypes.c_int64(0)
    budget = 2_000_000   # about 1 ms of SM clock
    rc = L.ludvig_debug_wait_timeout(budget, ctypes.byref(waited), None)
    assert rc == 4, ludvig.STATUS.get(rc)       # LUDVIG_ERR_TIMEOUT
    assert waited.value >= budget
    assert b"expired" in L.ludvig_last_error()
    # the context is intact: a tensor-core uplift still matches the oracle
    wl = inputs.small_field_workload(n=5000, views=2, d=40, width=61, height=45)
    sc = ludvig.Scene.from_inputs(wl.scene)
    out, beta = ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, device_features(wl, range(2)))
    torch.cuda.synchronize()
    f_ref, b_ref = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v))
    pos = b_ref > 0
    assert rel_l2(out.cpu().numpy(), f_ref, pos) <= 1e-5
    # a zero budget on a pending phase expires at once; arguments are checked
    assert L.ludvig_debug_wait_timeout(0, None, None) == 4
    assert L.ludvig_debug_wait_timeout(-1, None, None) == 1


@pytest.mark.parametrize("opt,k,code", [(ludvig.OPT_FAULT_LAUNCH, 7, "ERR_CUDA"), (ludvig.OPT_FAULT_ALLOC, 1, "ERR_OOM")])
def test_injected_host_faults_are_reported_and_recovered(opt, k, code):
    """A failure injected on the host (an allocation, a launch check) comes back
    as an error status with a message; the next call, with nothing armed,
    succeeds and matches the oracle."""
    wl = inputs.small_field_workload(n=4000, views=2, d=8, width=50, height=40)
    sc = ludvig.Scene.from_inputs(wl.scene)
    F = device_features(wl, range(2))
    ludvig.set_option(opt, k)
    try:
        with pytest.raises(ludvig.LudvigError, match=code) as ei:
            ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, F)
        assert "injected" in str(ei.value)
        assert ludvig.get_option(opt) == 0   # fired once, disarmed
    finally:
        ludvig.set_option(opt, 0)
    torch.cuda.synchronize()
    out, beta = ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, F)
    torch.cuda.synchronize()
    f_ref, b_ref = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v))
    pos = b_ref > 0
    assert rel_l2(out.cpu().numpy(), f_ref, pos) <= 1e-5
