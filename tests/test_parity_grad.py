"""Parity of simus_rf_grad (adjoint, FP32 on the CUDA cores) with the FP64 oracle's
analytic gradient (itself pinned by central finite differences in
test_oracle_pins.py), through the C ABI, and the autograd wrapper.

Tolerance: relative L2 error <= 1e-5 per gradient output (reflection coefficients, x,
z, delays), the FP32 budget; measured errors are ~1e-6.  Each gradient entry is a sum
over bins and transmits of oscillating products, reduced in a fixed order.
"""
import numpy as np
import pytest
import torch

from paper_2102_02738_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu
TOL_GRAD = 1e-5


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


def compare(S, oracle, w, seed=5):
    nt = w.cfg["n_samples"]
    drf = ph.normal(seed, 7, w.n_tx * w.cfg["n_elements"] * nt).reshape(w.n_tx, w.cfg["n_elements"], nt)
    drf = drf.astype(np.float32)
    gR, gx, gz, gd = oracle.rf_grad(w.cfg, w.delays, w.apod, w.x, None, w.z, w.rc, drf)
    plan = S.Plan(w.cfg)
    g = plan.rf_grad(*[dev(a) for a in (w.delays, w.apod, w.x, None, w.z, w.rc)], dev(drf))
    S.simus_plan_check(plan.handle)
    plan.close()
    errs = {"rc": rel_l2(g["rc"].cpu().numpy(), gR), "x": rel_l2(g["x"].cpu().numpy(), gx),
            "z": rel_l2(g["z"].cpu().numpy(), gz),
            "delays": rel_l2(g["delays"].cpu().numpy(), gd)}
    print(errs)
    return errs


@pytest.mark.parametrize("kw", [
    dict(n_elements=4, n_sub=2, n_scat=5, n_tx=2, nt=300),
    dict(n_elements=9, n_sub=3, n_scat=21, n_tx=3),
    dict(convex=True, n_elements=8, n_scat=12, n_tx=2),
    dict(baffle=1, n_elements=6, n_scat=10, n_tx=2),
    dict(baffle=2, n_elements=6, n_scat=10, n_tx=2),
    dict(n_elements=8, n_sub=2, n_scat=40, n_tx=14, nt=300),   # one lane per contraction item
])
def test_grad_tiny(S, oracle, kw):
    errs = compare(S, oracle, ph.tiny(**kw))
    assert max(errs.values()) <= TOL_GRAD


def test_grad_planewave_linear_128_reduced(S, oracle):
    """The 128-element 5 MHz 11-plane-wave geometry at 300 scatterers (the oracle's FP64
    gradient of the full 10,000-scatterer phantom takes minutes)."""
    errs = compare(S, oracle, ph.planewave_linear_128_grad(n_scat=300))
    assert max(errs.values()) <= TOL_GRAD


def test_grad_rejects_elevation(S):
    w = ph.tiny(y_spread=1e-3)
    plan = S.Plan(w.cfg)
    drf = torch.zeros(w.n_tx, w.cfg["n_elements"], w.cfg["n_samples"], device="cuda")
    with pytest.raises(S.SimusError) as ei:
        plan.rf_grad(*[dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)], drf)
    assert ei.value.code == -1


def test_grad_rejects_more_than_2048_channels(S):
    """T N > 2048 (transmit-element channels) is beyond the adjoint's shared-memory tiles:
    SIMUS_ERR_UNSUPPORTED before any launch; the forward path still runs."""
    w = ph.tiny(n_elements=160, n_sub=1, n_scat=10, n_tx=13, nt=300)
    plan = S.Plan(w.cfg)
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    drf = torch.zeros(w.n_tx, w.cfg["n_elements"], w.cfg["n_samples"], device="cuda")
    with pytest.raises(S.SimusError) as ei:
        plan.rf_grad(*args, drf)
    assert ei.value.code == -5
    rf = plan.rf(*args)
    torch.cuda.synchronize()
    assert torch.isfinite(rf).all()
    plan.close()


def test_autograd_misfit(S):
    """L = ||rf(x, z, R, tau) - rf_target||^2 through torch.autograd: the backward pass
    is simus_rf_grad with drf = 2 (rf - target)."""
    w = ph.planewave_linear_128_grad(n_scat=200)
    plan = S.Plan(w.cfg)
    tgt = plan.rf(*[dev(a) for a in (w.delays, w.apod)], dev(w.extra["x_target"]), None,
                  dev(w.extra["z_target"]), dev(w.rc))
    x = dev(w.x).requires_grad_()
    z = dev(w.z).requires_grad_()
    rc = dev(w.rc).requires_grad_()
    tau = dev(w.delays).requires_grad_()
    rf = S.rf_autograd(plan, x, z, rc, tau, dev(w.apod))
    loss = ((rf - tgt) ** 2).sum()
    loss.backward()
    drf = (2 * (rf.detach() - tgt)).contiguous()
    g = plan.rf_grad(tau.detach(), dev(w.apod), x.detach(), None, z.detach(), rc.detach(), drf)
    for name, t in (("x", x), ("z", z), ("rc", rc), ("delays", tau)):
        np.testing.assert_array_equal(t.grad.cpu().numpy(), g[name].cpu().numpy())
    assert loss.item() > 0
    plan.close()
