"""Failure detection without a GPU fault: every wait inside the library's kernels is
bounded, and a wait that gives up sets the plan's error flag, which simus_plan_check
reports as SIMUS_ERR_TIMEOUT while the device stays usable.  The self-test entry point
waits on a barrier phase that nothing completes (the failure is made on purpose, on the
host's request, and ends by itself after the stated number of polls)."""
import numpy as np
import pytest
import torch

from paper_2102_02738_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2102_02738_gb300 import build
    build.build()
    from paper_2102_02738_gb300 import simus
    return simus


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def test_bounded_wait_reports_timeout_and_device_stays_usable(S, oracle):
    w = ph.tiny(n_elements=16, n_scat=40, n_tx=3)
    plan = S.Plan(w.cfg, path="tc_f16")
    assert S.lib.simus_plan_check(plan.handle) == 0
    assert S.lib.simus_plan_selftest_timeout(plan.handle, 1 << 12, None) == 0
    assert S.lib.simus_plan_check(plan.handle) == -4                  # SIMUS_ERR_TIMEOUT
    assert b"bounded device wait" in S.lib.simus_last_error()
    assert S.lib.simus_plan_check(plan.handle) == 0                   # cleared
    # the context is intact: a tensor-core call right after gives the oracle's RF
    got = plan.rf(*[dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]).cpu().numpy()
    assert S.lib.simus_plan_check(plan.handle) == 0
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-3
    plan.close()


def test_selftest_rejects_bad_arguments(S):
    w = ph.tiny()
    plan = S.Plan(w.cfg)
    assert S.lib.simus_plan_selftest_timeout(plan.handle, 0, None) == -1
    assert S.lib.simus_plan_selftest_timeout(plan.handle, (1 << 24) + 1, None) == -1
    assert S.lib.simus_plan_selftest_timeout(None, 100, None) == -1
    plan.close()
