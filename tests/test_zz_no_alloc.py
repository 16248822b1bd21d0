"""simus_rf_noalloc, the allocation-free variant of simus_rf.  It serves callers that must
not allocate device memory: latency-critical loops that cannot enter an allocator (which
may synchronise the device), and plug-ins whose host application owns the device memory.
It keeps its temporaries in a fixed per-device array instead of a plan's workspace.  This
file is collected last on purpose.

Checks, through the C ABI:
- two calls in a row on different problems each match the FP64 oracle within the FP32
  tolerance (relative L2 <= 1e-5), and simus_rf on a plain FP32 plan;
- the first problem's partial spectra do not fit the array at the chunk count simus_rf
  would use, so the call takes the route with fewer, longer scatterer chunks;
- a stream under capture is refused before any device work;
- a problem whose temporaries exceed the fixed array is rejected before any device work.
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


def no_alloc(S, w, stream=None):
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    out = torch.full((w.n_tx, w.cfg["n_elements"], w.cfg["n_samples"]), float("nan"),
                     device="cuda")
    S.simus_rf_noalloc(w.cfg, w.cfg["n_samples"], *args, out, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_two_calls_in_a_row_match_the_oracle(S, oracle):
    # 96 elements x 44 transmits x 206 bins: a partial spectrum is ~7 MB, so the 32 MiB
    # array holds two chunks where the plain launch shape would use three
    first = ph.tiny(n_elements=96, n_sub=2, n_scat=400, n_tx=44)
    second = ph.tiny(n_elements=24, n_sub=2, n_scat=203, n_tx=3, y_spread=1e-3)
    got1 = no_alloc(S, first)
    got2 = no_alloc(S, second)
    ref1 = oracle.rf(first.cfg, first.delays, first.apod, first.x, first.y, first.z, first.rc)
    ref2 = oracle.rf(second.cfg, second.delays, second.apod, second.x, second.y, second.z,
                     second.rc)
    assert rel_l2(got1, ref1) <= TOL_F32
    assert rel_l2(got2, ref2) <= TOL_F32
    # and the same RF as the plan-based entry point
    assert rel_l2(got1, with_plan(S, first)) <= TOL_F32
    assert rel_l2(got2, with_plan(S, second)) <= TOL_F32


def test_stream_capture_is_refused(S):
    w = ph.tiny(n_elements=8, n_scat=20, n_tx=2)
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    out = torch.zeros((w.n_tx, 8, w.cfg["n_samples"]), device="cuda")
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        with pytest.raises(S.SimusError) as ei:
            S.simus_rf_noalloc(w.cfg, w.cfg["n_samples"], *args, out, st)
    assert ei.value.code == -1 and b"capture" in S.lib.simus_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    # the entry point still works on an ordinary stream afterwards
    ref = with_plan(S, w)
    assert rel_l2(no_alloc(S, w), ref) <= TOL_F32


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
