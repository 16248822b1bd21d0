"""Parity of the CUDA RF path with the FP64 oracle, element by element, on the same
seeded float32 inputs, through the C ABI.

Tolerance (stated by the method's accuracy target): relative L2 error
||gpu - oracle|| / ||oracle|| <= 1e-5 for the FP32 path over the compared outputs.
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


def gpu_rf(S, w, path="plain", spectrum=False):
    plan = S.Plan(w.cfg, path=path)
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    out = plan.rf_spectrum(*args) if spectrum else plan.rf(*args)
    torch.cuda.synchronize()
    info = plan.info
    plan.close()
    return out.cpu().numpy(), info


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_plan_bins_match_oracle(S, oracle):
    for w in (ph.focused_linear_64(), ph.planewave_linear_128(n_scat=10),
              ph.diverging_convex_128(n_scat=10, n_tx=2), ph.tiny(pulse=1)):
        plan = S.Plan(w.cfg)
        lo, hi, n = oracle.bins(w.cfg)
        assert (plan.info["q_lo"], plan.info["q_hi"], plan.info["n_bins"]) == (lo, hi, n)
        assert plan.info["n_sub"] == oracle.nsub(w.cfg)
        plan.close()


@pytest.mark.parametrize("kw", [
    dict(),                                            # linear, soft baffle, nu = 2
    dict(n_sub=1, n_tx=3),
    dict(n_sub=3, n_elements=7, n_scat=37),            # ragged scatterer groups
    dict(convex=True, n_elements=8),
    dict(baffle=1), dict(baffle=2),
    dict(pulse=1, alpha_db=0.0),
    dict(y_spread=1.5e-3),                             # scatterers off the azimuth plane
    dict(elev_focus=float("inf")),
    dict(n_elements=24, n_scat=150, n_tx=7),           # one Green's tile for all transmits
    dict(convex=True, n_elements=11, n_scat=60, n_tx=5),  # odd N: the last element pair half empty
    dict(n_elements=24, n_scat=70, n_tx=7, y_spread=1e-3),
    dict(n_elements=48, n_scat=40, n_tx=45),           # T N = 2160: smaller scatterer groups
    dict(n_elements=96, n_scat=12, n_tx=70),           # T N = 6720: per-transmit tiles
])
def test_rf_tiny_configs(S, oracle, kw):
    w = ph.tiny(**kw)
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    got, _ = gpu_rf(S, w)
    assert got.shape == ref.shape
    assert rel_l2(got, ref) <= TOL_F32


def test_rf_focused_linear_64_full(S, oracle):
    """64-element 5 MHz focused transmit, 200 scatterers: the whole RF, every sample."""
    w = ph.focused_linear_64()
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    got, info = gpu_rf(S, w)
    assert info["n_bins"] > 16 * 10          # spans many bin tiles
    assert rel_l2(got, ref) <= TOL_F32


def test_spectrum_many_tiles_ragged(S, oracle):
    """Sizes spanning several bin tiles and scatterer chunks with ragged tails."""
    w = ph.tiny(n_elements=24, n_sub=2, n_scat=203, n_tx=2, nt=1001)
    lo, hi, n = oracle.bins(w.cfg)
    assert n % 16 != 0
    ref = oracle.rf_spectrum(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc, np.arange(lo, hi + 1))
    got, _ = gpu_rf(S, w, spectrum=True)
    assert rel_l2(got, ref) <= TOL_F32


def test_spectrum_planewave_linear_128_sampled_bins(S, oracle):
    """Full-size 128-element nu = 3 plane wave, 20,003 scatterers, in the configuration the
    benchmark times: spectra compared at sampled bins the oracle computes one by one."""
    w = ph.planewave_linear_128()
    got, info = gpu_rf(S, w, spectrum=True)
    lo = info["q_lo"]
    ks = np.array([0, 97, info["n_bins"] // 2, info["n_bins"] - 1])
    ref = oracle.rf_spectrum(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc, lo + ks)
    assert rel_l2(got[..., ks], ref) <= TOL_F32


def test_linearity_full_size(S):
    """RF is linear in the reflection coefficients (any size)."""
    w = ph.planewave_linear_128()
    a, _ = gpu_rf(S, w)
    w2 = ph.planewave_linear_128()
    w2.rc = (2.0 * w.rc).astype(np.float32)      # exact in float32
    b, _ = gpu_rf(S, w2)
    np.testing.assert_array_equal(b, 2.0 * a)


def test_deterministic(S):
    w = ph.tiny(n_elements=16, n_scat=300)
    a, _ = gpu_rf(S, w)
    b, _ = gpu_rf(S, w)
    np.testing.assert_array_equal(a, b)


def test_empty_scatterers_give_zeros(S):
    w = ph.tiny()
    w.x, w.z, w.rc = (np.zeros(0, np.float32),) * 3
    plan = S.Plan(w.cfg)
    d = [dev(a) for a in (w.delays, w.apod)]
    e = torch.zeros(0, device="cuda")
    out = torch.full((w.n_tx, w.cfg["n_elements"], w.cfg["n_samples"]), 7.0, device="cuda")
    plan.rf(*d, e, None, e, e, out=out)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


def test_errors_are_reported(S):
    w = ph.tiny()
    plan = S.Plan(w.cfg)
    d = [dev(a) for a in (w.delays, w.apod, w.x, None, w.z, w.rc)]
    host = torch.zeros(w.n_tx, w.cfg["n_elements"], w.cfg["n_samples"])
    with pytest.raises(TypeError):
        plan.rf(*d, out=host)          # binding refuses a host tensor
    bad = S.Tx(w.n_tx, 0, d[0].data_ptr(), None)
    import ctypes as C
    rc = S.lib.simus_rf(plan.handle, C.byref(bad), C.byref(S.scat_struct(*d[2:])),
                        C.c_void_p(torch.empty(1, device="cuda").data_ptr()), None)
    assert rc == -1 and b"apod" in S.lib.simus_last_error()
