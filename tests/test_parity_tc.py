"""Parity of the batched tensor-core path (FP16 / BF16 operands on tcgen05, FP32
accumulation) with the FP64 oracle, through the C ABI.

Tolerance: relative L2 error <= 2e-3 over the compared outputs (the accuracy target of
the reduced-precision contraction); the FP32 Green's-term generation is shared with the
plain path, whose own tolerance is 1e-5.  The BF16 path carries every operand as a BF16
leading part and a BF16 remainder (three products per GEMM), which takes arrays of up to
176 elements.
"""
import numpy as np
import pytest
import torch

from paper_2102_02738_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu
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


def run(S, w, path, spectrum=False):
    plan = S.Plan(w.cfg, path=path)
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    out = plan.rf_spectrum(*args) if spectrum else plan.rf(*args)
    S.lib.simus_plan_check(plan.handle) == 0 or pytest.fail(S.lib.simus_last_error().decode())
    out = out.cpu().numpy()
    info = plan.info
    plan.close()
    return out, info


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


TINY = [
    dict(),
    dict(n_elements=16, n_scat=300, n_tx=5),                 # several scatterer tiles
    dict(n_elements=13, n_sub=3, n_scat=150, n_tx=3),        # N not a multiple of 8
    dict(convex=True, n_elements=24, n_scat=200, n_tx=9),
    dict(y_spread=1e-3, n_scat=130),
    dict(convex=True, n_elements=24, n_scat=300, n_tx=5, y_spread=2e-3),   # Y != 0, convex
    dict(n_elements=13, n_sub=3, n_scat=150, n_tx=3, y_spread=1.5e-3),     # Y != 0, odd N
    # wide arrays: 96-112 KB tiles leave room for one shared-memory tile buffer, so the
    # later bins of a pass wait in tensor-memory stash slots
    dict(n_elements=176, n_sub=1, n_scat=140, n_tx=3),      # two buffers, receive in halves
    dict(n_elements=200, n_sub=1, n_scat=140, n_tx=3),      # one buffer, two stash slots
    dict(n_elements=256, n_sub=1, n_scat=140, n_tx=2),      # one buffer, one stash slot
    dict(n_elements=200, n_sub=1, n_scat=60, n_tx=21),      # large T x N: one bin per pass
]


@pytest.mark.parametrize("kw", TINY)
def test_tc_f16_rf_tiny(S, oracle, kw):
    w = ph.tiny(**kw)
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    got, _ = run(S, w, "tc_f16")
    assert rel_l2(got, ref) <= TOL_TC


@pytest.mark.parametrize("kw", [kw for kw in TINY if kw.get("n_elements", 4) <= 176] + [
    dict(n_elements=170, n_sub=1, n_scat=300, n_tx=9),      # split tile near its width limit
    dict(n_elements=64, n_sub=2, n_scat=700, n_tx=31),      # two transmit groups of 16
])
def test_tc_bf16_rf_tiny(S, oracle, kw):
    """BF16 leading parts + remainders: within the reduced-precision budget."""
    w = ph.tiny(**kw)
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    got, _ = run(S, w, "tc_bf16")
    err = rel_l2(got, ref)
    print(f"bf16 rel-L2 {err:.3e}")
    assert err <= TOL_TC


def test_tc_f16_matches_plain_spectrum(S):
    """Same Green's terms, different contraction precision: the two GPU paths agree to
    the FP16 budget on a case with many bin tiles and scatterer tiles."""
    w = ph.tiny(n_elements=64, n_sub=2, n_scat=1000, n_tx=12, nt=900)
    a, _ = run(S, w, "plain", spectrum=True)
    b, _ = run(S, w, "tc_f16", spectrum=True)
    assert rel_l2(b, a) <= TOL_TC


def test_tc_bf16_meets_the_reduced_precision_budget(S, oracle):
    """Rounding G, the transmit weights, R P and G again to BF16 (8-bit significand) would
    give ~3.2e-3 on this case (four roundings of ~1.6e-3 each); with the remainders the
    contraction carries ~16 significant bits."""
    w = ph.tiny(n_elements=32, n_scat=400, n_tx=7)
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    got, _ = run(S, w, "tc_bf16")
    err = rel_l2(got, ref)
    print(f"bf16 rel-L2 {err:.3e}")
    assert err <= TOL_TC


@pytest.mark.parametrize("pair", [0, 1])
def test_tc_bf16_pass_modes(S, oracle, pair):
    """Split BF16 with one-bin (pair 0) and two-bin (pair 1, one stash slot of 2 Np
    columns) generation passes, set through the tuning interface."""
    w = ph.tiny(convex=True, n_elements=24, n_scat=400, n_tx=9)
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    plan = S.Plan(w.cfg, path="tc_bf16")
    plan.set_tuning(pair=pair, max_bins=4)
    got = plan.rf(*[dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]).cpu().numpy()
    assert S.lib.simus_plan_check(plan.handle) == 0
    plan.close()
    assert rel_l2(got, ref) <= TOL_TC


def test_tc_bf16_rejects_arrays_wider_than_the_split_tile(S):
    """The leading-part and remainder tiles of more than 176 elements do not fit one
    CTA's shared memory: SIMUS_ERR_UNSUPPORTED before any launch; FP16 takes them."""
    w = ph.tiny(n_elements=200, n_sub=1, n_scat=20, n_tx=2, nt=300)
    plan = S.Plan(w.cfg, path="tc_bf16")
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    with pytest.raises(S.SimusError) as ei:
        plan.rf(*args)
    assert ei.value.code == -5
    plan.close()
    got, _ = run(S, w, "tc_f16")
    assert np.isfinite(got).all() and np.abs(got).max() > 0


def test_tc_rejects_arrays_wider_than_256_elements(S):
    """More than 256 elements do not fit one CTA's operands: the call fails before any
    launch with SIMUS_ERR_UNSUPPORTED and the plan and the context stay usable."""
    w = ph.tiny(n_elements=264, n_sub=1, n_scat=20, n_tx=2, nt=300)
    plan = S.Plan(w.cfg, path="tc_f16")
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    with pytest.raises(S.SimusError) as ei:
        plan.rf(*args)
    assert ei.value.code == -5
    plan.close()
    ok = ph.tiny(n_elements=8, n_scat=20, n_tx=2)
    got, _ = run(S, ok, "tc_f16")
    assert np.isfinite(got).all() and np.abs(got).max() > 0


@pytest.mark.parametrize("path", ["tc_f16", "tc_bf16"])
def test_tc_diverging_convex_128_sampled_bins(S, oracle, path):
    """Full-size 128-element convex array, 31 diverging waves, 100,000 scatterers, in the
    launch configuration the benchmark times: spectra at sampled bins vs the oracle."""
    w = ph.diverging_convex_128()
    got, info = run(S, w, path, spectrum=True)
    lo = info["q_lo"]
    ks = np.array([3, info["n_bins"] // 2, info["n_bins"] - 2])
    ref = oracle.rf_spectrum(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc, lo + ks)
    err = rel_l2(got[..., ks], ref)
    print(f"{path} rel-L2 {err:.3e}")
    assert err <= TOL_TC


def test_tc_linearity(S):
    w = ph.tiny(n_elements=32, n_scat=500, n_tx=4)
    a, _ = run(S, w, "tc_f16")
    w.rc = (2.0 * w.rc).astype(np.float32)
    b, _ = run(S, w, "tc_f16")
    # FP16 rounding of 2 R P equals 2 x the rounding of R P (power-of-two scale)
    np.testing.assert_allclose(b, 2.0 * a, rtol=0, atol=1e-6 * np.abs(a).max())
