"""Parity of the 2-D mode (Section V, Eq. 36-38: Green's term exp(i(k + i k_a) r)/sqrt(r)
times D, no elevation factor) with the FP64 oracle, through the C ABI: plain FP32 RF
(tolerance 1e-5), tensor-core FP16 RF (2e-3), RMS field (1e-5), adjoint gradients (1e-5),
a batch that mixes 2-D and 3-D simulations, and the rejection of an elevation coordinate.
"""
import numpy as np
import pytest
import torch

from paper_2102_02738_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu
TOL_F32 = 1e-5
TOL_TC = 2e-3


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


def gpu_rf(S, w, path):
    plan = S.Plan(w.cfg, path=path)
    out = plan.rf(*[dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]).cpu().numpy()
    assert S.lib.simus_plan_check(plan.handle) == 0
    plan.close()
    return out


CASES = [dict(), dict(n_sub=3, n_elements=7, n_scat=37, n_tx=3),
         dict(convex=True, n_elements=8, n_scat=20), dict(baffle=1, n_scat=9),
         dict(baffle=2, n_elements=6, n_scat=11), dict(n_elements=16, n_scat=300, n_tx=5)]


@pytest.mark.parametrize("kw", CASES)
def test_two_d_plain_rf(S, oracle, kw):
    w = ph.tiny(two_d=True, **kw)
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, None, w.z, w.rc)
    assert rel_l2(gpu_rf(S, w, "plain"), ref) <= TOL_F32


@pytest.mark.parametrize("kw", CASES)
def test_two_d_tc_rf(S, oracle, kw):
    w = ph.tiny(two_d=True, **kw)
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, None, w.z, w.rc)
    assert rel_l2(gpu_rf(S, w, "tc_f16"), ref) <= TOL_TC


def test_two_d_differs_from_three_d(S):
    w3 = ph.tiny(n_scat=20)
    w2 = ph.tiny(n_scat=20, two_d=True)
    a, b = gpu_rf(S, w3, "plain"), gpu_rf(S, w2, "plain")
    assert rel_l2(a / np.abs(a).max(), b / np.abs(b).max()) > 1e-2


def test_two_d_pfield(S, oracle):
    w = ph.tiny(two_d=True, n_tx=2, convex=True, n_elements=8)
    X, Z = np.meshgrid(np.linspace(-4e-3, 4e-3, 9), np.linspace(2e-3, 14e-3, 7))
    x, z = X.ravel().astype(np.float32), Z.ravel().astype(np.float32)
    cfg = w.cfg
    xe, ze = ph.element_centres(cfg)
    r_max = float(np.max(np.hypot(x[:, None] - xe[None, :], z[:, None] - ze[None, :]))) + cfg["width"]
    nf = S.simus_pfield_nfreq(cfg, r_max, float(w.delays.max()))
    plan = S.Plan(cfg)
    got = plan.pfield(dev(w.delays), dev(w.apod), dev(x), None, dev(z), nf).cpu().numpy()
    plan.close()
    ref = oracle.pfield(cfg, w.delays, w.apod, x, None, z, nf)
    assert rel_l2(got, ref) <= TOL_F32


@pytest.mark.parametrize("kw", [dict(n_elements=4, n_sub=2, n_scat=5, n_tx=2, nt=300),
                                dict(convex=True, n_elements=8, n_scat=12, n_tx=2)])
def test_two_d_gradients(S, oracle, kw):
    w = ph.tiny(two_d=True, **kw)
    nt = w.cfg["n_samples"]
    drf = ph.normal(5, 7, w.n_tx * w.cfg["n_elements"] * nt).reshape(w.n_tx, w.cfg["n_elements"], nt)
    drf = drf.astype(np.float32)
    gR, gx, gz, gd = oracle.rf_grad(w.cfg, w.delays, w.apod, w.x, None, w.z, w.rc, drf)
    plan = S.Plan(w.cfg)
    g = plan.rf_grad(*[dev(a) for a in (w.delays, w.apod, w.x, None, w.z, w.rc)], dev(drf))
    assert S.lib.simus_plan_check(plan.handle) == 0
    plan.close()
    for got, ref in ((g["rc"], gR), (g["x"], gx), (g["z"], gz), (g["delays"], gd)):
        assert rel_l2(got.cpu().numpy(), ref) <= TOL_F32


def test_batch_mixes_two_d_and_three_d(S, oracle):
    sims = [ph.tiny(two_d=True, n_elements=12, n_scat=150, n_tx=3, seed=11),
            ph.tiny(n_elements=12, n_scat=150, n_tx=3, seed=12),
            ph.tiny(two_d=True, convex=True, n_elements=10, n_scat=80, n_tx=2, seed=13)]
    plans = [S.Plan(w.cfg, path="tc_f16") for w in sims]
    txs = [(dev(w.delays), dev(w.apod)) for w in sims]
    scs = [(dev(w.x), None, dev(w.z), dev(w.rc)) for w in sims]
    rfs = [torch.empty((w.n_tx, w.cfg["n_elements"], w.cfg["n_samples"]), device="cuda") for w in sims]
    S.simus_batch_rf([p.handle for p in plans], txs, scs, rfs)
    for w, rf in zip(sims, rfs):
        ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, None, w.z, w.rc)
        assert rel_l2(rf.cpu().numpy(), ref) <= TOL_TC
    for p in plans:
        p.close()


def test_two_d_rejects_elevation(S):
    w = ph.tiny(two_d=True, y_spread=1e-3)
    plan = S.Plan(w.cfg)
    with pytest.raises(S.SimusError) as ei:
        plan.rf(*[dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)])
    assert ei.value.code == -1 and "2-D" in S.lib.simus_last_error().decode()
    plan.close()
