"""Parity of simus_pfield (RMS pressure field, Eq. 22 and Eq. 41-42, FP32) with the FP64
oracle on the same seeded points, through the C ABI.  Tolerance: relative L2 <= 1e-5.

Includes coarse versions of the paper's two field examples: the focused 64-element
2.7 MHz P4-2v cardiac array (Fig. 9 caption parameters) and the 128-element 7.6 MHz
L11-5v linear array with a 10-degree plane wave (Fig. 10 caption parameters).
"""
import math

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


def grid(x0, x1, nx, z0, z1, nz, y=None):
    X, Z = np.meshgrid(np.linspace(x0, x1, nx), np.linspace(z0, z1, nz))
    Y = None if y is None else np.full(X.size, y)
    return X.ravel().astype(np.float32), (None if Y is None else Y.astype(np.float32)), \
        Z.ravel().astype(np.float32)


def run(S, oracle, cfg, delays, apod, x, y, z):
    xe, ze = ph.element_centres(cfg)
    r_max = float(np.max(np.hypot(x[:, None] - xe[None, :], z[:, None] - ze[None, :]))) + cfg["width"]
    nf = S.simus_pfield_nfreq(cfg, r_max, float(delays.max()))
    assert nf == oracle.pfield_nfreq(cfg, r_max, float(delays.max()))
    plan = S.Plan(cfg)
    got = plan.pfield(dev(delays), dev(apod), dev(x), dev(y), dev(z), nf).cpu().numpy()
    S.simus_plan_check(plan.handle)
    plan.close()
    ref = oracle.pfield(cfg, delays, apod, x, y, z, nf)
    return got, ref


@pytest.mark.parametrize("kw,y", [(dict(n_tx=2), None), (dict(convex=True, n_elements=8), None),
                                  (dict(n_sub=3, baffle=2), 0.8e-3)])
def test_pfield_tiny(S, oracle, kw, y):
    w = ph.tiny(**kw)
    x, yy, z = grid(-4e-3, 4e-3, 9, 2e-3, 14e-3, 7, y)
    got, ref = run(S, oracle, w.cfg, w.delays, w.apod, x, yy, z)
    assert rel_l2(got, ref) <= TOL_F32


def test_pfield_p4_2v_focused(S, oracle):
    """Fig. 9 setup: 64 elements, 2.7 MHz, pitch 0.3 mm, kerf 50 um, 74 % bandwidth,
    elevation focus 6 cm; focused at 6 cm depth; coarse x-z grid to 10 cm."""
    probe = ph.linear_probe(64, 2.7e6, 0.30e-3, 0.05e-3, elev_focus=0.06, frac_bw=0.74)
    cfg = dict(probe, **ph.medium(2.7e6), n_samples=64)
    delays = ph.focused_delays(probe, cfg["c"], 0.0, 0.06).astype(np.float32)
    apod = np.ones_like(delays)
    x, y, z = grid(-2e-2, 2e-2, 21, 5e-3, 0.1, 19)
    got, ref = run(S, oracle, cfg, delays, apod, x, y, z)
    assert rel_l2(got, ref) <= TOL_F32
    # the beam is centred: at the focal depth the lateral RMS profile peaks on the axis
    zz = np.linspace(5e-3, 0.1, 19)
    row = got[0].reshape(19, 21)[np.argmin(np.abs(zz - 0.06))]
    assert np.argmax(row) == 10


def test_pfield_l11_5v_tilted_plane_wave(S, oracle):
    """Fig. 10 setup: 128 elements, 7.6 MHz, pitch 0.27 mm, kerf 30 um, 77 % bandwidth,
    elevation focus 1.8 cm; plane wave tilted by 10 degrees; coarse grid to 3 cm."""
    probe = ph.linear_probe(128, 7.6e6, 0.27e-3, 0.03e-3, elev_focus=0.018, frac_bw=0.77)
    cfg = dict(probe, **ph.medium(7.6e6), n_samples=64)
    delays = ph.plane_wave_delays(probe, cfg["c"], [math.radians(10)]).astype(np.float32)
    apod = np.ones_like(delays)
    x, y, z = grid(-1.5e-2, 2.0e-2, 15, 3e-3, 3e-2, 12)
    got, ref = run(S, oracle, cfg, delays, apod, x, y, z)
    assert rel_l2(got, ref) <= TOL_F32
