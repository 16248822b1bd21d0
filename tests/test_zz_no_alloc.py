"""simus_rf_noalloc, the allocation-free variant of simus_rf for callers that cannot
allocate device memory (stream capture in global mode, allocator-free real-time loops,
plug-ins whose host owns the device memory).  It keeps its temporaries in a fixed
per-device array instead of a plan's workspace.  This file is collected last on purpose.

Checks, through the C ABI: two calls in a row on different problems each match
simus_rf on a plain FP32 plan within the FP32 tolerance (relative L2 <= 1e-5), and a
problem whose temporaries exceed the fixed array is rejected before any device work.
"""

import numpy as np
import pytest
import torch

from paper_2102_02738_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu
TOL_F32 = 1e-5


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


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def with_plan(S, w):
    plan = S.Plan(w.cfg, path="plain")
    out = plan.rf(*[dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)])
    torch.cuda.synchronize()
    plan.close()
    return out.cpu().numpy()


def no_alloc(S, w):
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    out = torch.full((w.n_tx, w.cfg["n_elements"], w.cfg["n_samples"]), float("nan"),
                     device="cuda")
    S.simus_rf_noalloc(w.cfg, w.cfg["n_samples"], *args, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_two_calls_in_a_row_match_simus_rf(S):
    first = ph.planewave_linear_128(n_scat=3000)                     # fills many chunks
    second = ph.tiny(n_elements=24, n_sub=2, n_scat=203, n_tx=3, y_spread=1e-3)
    got1 = no_alloc(S, first)
    got2 = no_alloc(S, second)
    assert rel_l2(got1, with_plan(S, first)) <= TOL_F32
    assert rel_l2(got2, with_plan(S, second)) <= TOL_F32


def test_oversized_problem_is_rejected(S):
    w = ph.planewave_linear_128(n_scat=8)
    w.delays = np.repeat(w.delays, 64, axis=0)                       # 64 transmits
    w.apod = np.repeat(w.apod, 64, axis=0)
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    out = torch.zeros((64, 128, w.cfg["n_samples"]), device="cuda")
    with pytest.raises(S.SimusError) as ei:
        S.simus_rf_noalloc(w.cfg, w.cfg["n_samples"], *args, out)
    assert ei.value.code == -1 and b"scratch" in S.lib.simus_last_error()
    assert torch.count_nonzero(out).item() == 0
