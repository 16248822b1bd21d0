"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check compares the oracle with something other than itself: printed values
(tests/golden/), closed forms, numerical quadrature of the defining integrals,
invariants (reciprocity, linearity, superposition), a library routine (numpy's FFT),
the brute-force aperture integral, and finite differences.  A dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from paper_2102_02738_gb300 import phantoms as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cfg(**kw):
    w = ph.tiny(**kw)
    return w


def quad_c(fn, a, b, **kw):
    re = integrate.quad(lambda t: fn(t).real, a, b, limit=400, **kw)[0]
    im = integrate.quad(lambda t: fn(t).imag, a, b, limit=400, **kw)[0]
    return re + 1j * im


# ------------------------------------------------------------------------- Eq. 18
def test_gaussian_coefficients_are_the_printed_ones(oracle):
    rows = np.loadtxt(os.path.join(GOLDEN, "eq18_gaussian_coefficients.txt"))
    A, B = oracle.gaussian_coefficients()
    np.testing.assert_array_equal(A.real, rows[:, 1])
    np.testing.assert_array_equal(A.imag, rows[:, 2])
    np.testing.assert_array_equal(B.real, rows[:, 3])
    np.testing.assert_array_equal(B.imag, rows[:, 4])
    # the sum of Gaussians approximates the rectangle Pi(u) (Eq. 12, Fig. 5)
    u = np.linspace(-2, 2, 4001)
    v = (A[:, None] * np.exp(-B[:, None] * u**2)).sum(0)
    assert np.abs(v.imag).max() < 1e-12                    # conjugate pairs: real sum
    inside, outside = np.abs(u) < 0.45, np.abs(u) > 0.55
    assert np.abs(v.real[inside] - 1).max() < 0.11
    assert np.abs(v.real[outside]).max() < 0.09
    assert np.sqrt(np.trapezoid((v.real - (np.abs(u) < 0.5)) ** 2, u)) < 0.15


# ------------------------------------------------------------------ Eq. 26-27, App. B
@pytest.mark.parametrize("bw", [0.5, 0.65, 0.75, 0.77, 1.0])
def test_transducer_response_appendix_b(oracle, bw):
    cfg = _cfg().cfg
    cfg["frac_bw"] = bw
    wc = 2 * np.pi * cfg["fc"]
    wb = bw * wc
    S = oracle.transducer_response(cfg, [wc, wc - wb / 2, wc + wb / 2, 0.0, 2 * wc])
    assert S[0] == pytest.approx(1.0, abs=1e-15)
    assert S[1] == pytest.approx(0.5, rel=1e-12)           # -6 dB two-way (Eq. 47)
    assert S[2] == pytest.approx(0.5, rel=1e-12)
    assert S[3] == pytest.approx(2.0**-126, rel=1e-9)      # Eq. 49
    assert S[4] == pytest.approx(2.0**-126, rel=1e-9)


def test_fig8_bandwidth_example(oracle):
    """Fig. 8: 77 % bandwidth at 7.6 MHz has its two-way -6 dB points at fc(1 +- 0.385)."""
    cfg = _cfg(fc=7.6e6).cfg
    cfg["frac_bw"] = 0.77
    f = np.array([7.6e6 * (1 - 0.385), 7.6e6 * (1 + 0.385)])
    np.testing.assert_allclose(20 * np.log10(oracle.transducer_response(cfg, 2 * np.pi * f)),
                               20 * np.log10(0.5), rtol=1e-9)


# ------------------------------------------------------------------------- Eq. 25
@pytest.mark.parametrize("pulse,cycles", [(0, 1.0), (0, 2.5), (1, 1.0), (1, 3.0)])
def test_pulse_spectrum_is_fourier_transform_of_windowed_sine(oracle, pulse, cycles):
    cfg = _cfg(pulse=pulse).cfg
    cfg["pulse_cycles"] = cycles
    fc = cfg["fc"]
    wc, T = 2 * np.pi * fc, cycles / fc

    def window(t):
        return 1.0 if pulse == 0 else 0.5 * (1 + math.cos(2 * math.pi * t / T))

    for w in wc * np.array([0.2, 0.7, 1.0, 1.3, 1.9]):
        ft = quad_c(lambda t: math.sin(wc * t) * window(t) * np.exp(1j * w * t), -T / 2, T / 2)
        sp = oracle.pulse_spectrum(cfg, w)[0]
        # Eq. 25 equals (2/T) * FT with the e^{+i w t} kernel of the Eq. 1 convention
        assert sp == pytest.approx(2 / T * ft, rel=1e-9, abs=1e-12)


# ------------------------------------------------------------------------- Eq. 21
def test_nsub_matches_paper_typical_values(oracle):
    with open(os.path.join(GOLDEN, "probe_examples.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    for name, N, fc, pitch, kerf, bw, rf, nu in rows:
        probe = ph.linear_probe(int(N), float(fc), float(pitch), float(kerf),
                                elev_focus=float(rf), frac_bw=float(bw))
        cfg = dict(probe, **ph.medium(float(fc)), n_samples=1000)
        assert oracle.nsub(cfg) == int(nu), name


def test_nsub_sub_element_not_wider_than_lambda_min(oracle):
    for fc in (2e6, 3e6, 5e6, 7.6e6, 12e6):
        for pitch in (0.1e-3, 0.2e-3, 0.3e-3, 0.5e-3):
            cfg = dict(ph.linear_probe(64, fc, pitch, 0.02e-3), **ph.medium(fc), n_samples=100)
            nu = oracle.nsub(cfg)
            lam_min = cfg["c"] / (fc * (1 + cfg["frac_bw"] / 2))
            assert cfg["width"] / nu <= lam_min * (1 + 1e-12)
            assert nu == 1 or cfg["width"] / (nu - 1) > lam_min


# ------------------------------------------------------------------ bin selection
def test_bins_are_exactly_the_above_threshold_range(oracle):
    for w in (ph.focused_linear_64(), ph.tiny(nt=300), ph.tiny(pulse=1, nt=512)):
        cfg = w.cfg
        nt = cfg["n_samples"]
        q = np.arange(1, (nt - 1) // 2 + 1)
        H = np.abs(oracle.transfer(cfg, 2 * np.pi * q * cfg["fs"] / nt))
        keep = q[H >= 1e-5 * H.max()]
        lo, hi, n = oracle.bins(cfg)
        assert (lo, hi, n) == (keep.min(), keep.max(), keep.max() - keep.min() + 1)
        assert np.array_equal(keep, np.arange(lo, hi + 1))   # contiguous


# ------------------------------------------------------------------------ Eq. 24
def test_linear_centroids_eq24(oracle):
    for nu in (1, 2, 3, 5):
        cfg = _cfg(n_elements=6, n_sub=nu).cfg
        xc, zc, psi = oracle.centroids(cfg)
        N, p, b = 6, cfg["pitch"], cfg["width"] / 2
        assert len(xc) == nu * N and np.all(zc == 0) and np.all(psi == 0)
        centres = xc.reshape(N, nu).mean(1)
        np.testing.assert_allclose(centres, (np.arange(N) - (N - 1) / 2) * p, atol=1e-15)
        np.testing.assert_allclose(np.diff(xc.reshape(N, nu), axis=1), 2 * b / nu, rtol=1e-12)
        np.testing.assert_allclose(xc.reshape(N, nu)[:, 0] - centres, -b + b / nu, atol=1e-15)
        assert np.all(np.diff(xc) > 0)                        # numbered left to right


def test_convex_centroids_on_arc(oracle):
    cfg = _cfg(n_elements=8, n_sub=2, convex=True).cfg
    xc, zc, psi = oracle.centroids(cfg)
    R = cfg["radius"]
    np.testing.assert_allclose(np.hypot(xc, zc + R), R, rtol=1e-14)
    np.testing.assert_allclose(psi, np.arctan2(xc, zc + R), atol=1e-14)
    ang_el = psi.reshape(8, 2).mean(1)
    np.testing.assert_allclose(np.diff(ang_el) * R, cfg["pitch"], rtol=1e-12)
    np.testing.assert_allclose(ang_el.mean(), 0.0, atol=1e-15)


def test_convex_scatterer_on_normal_sees_broadside(oracle):
    cfg = _cfg(n_elements=8, n_sub=2, convex=True, alpha_db=0.0).cfg
    xc, zc, psi = oracle.centroids(cfg)
    n, d, f = 5, 7e-3, 4e6
    X, Z = xc[n] + d * math.sin(psi[n]), zc[n] + d * math.cos(psi[n])
    k = 2 * math.pi * f / cfg["c"]
    g = oracle.green(cfg, f, X, 0.0, Z, n)
    expect = np.exp(1j * k * d) / d * oracle.delta(cfg, k, 0.0, d)   # D = 1 on the normal
    assert g == pytest.approx(expect, rel=1e-12)


# ------------------------------------------------------------------------- Eq. 10, 39
def test_directivity_is_aperture_integral(oracle):
    cfg = _cfg(baffle=1).cfg
    k, b = 2 * math.pi * 6e6 / 1540, 0.2e-3
    for st in (0.0, 0.1, -0.4, 0.8, 0.99):
        ct = math.sqrt(1 - st * st)
        integ = quad_c(lambda x: np.exp(-1j * k * x * st), -b, b)
        assert oracle.directivity(cfg, k, b, st, ct) == pytest.approx(integ.real / (2 * b), abs=1e-12)
        assert abs(integ.imag) < 1e-15
        soft = dict(cfg, baffle=0)
        imp = dict(cfg, baffle=2, zeta=1.75)
        d = integ.real / (2 * b)
        assert oracle.directivity(soft, k, b, st, ct) == pytest.approx(d * ct, abs=1e-12)
        assert oracle.directivity(imp, k, b, st, ct) == pytest.approx(d * ct / (ct + 1.75), abs=1e-12)
    assert oracle.directivity(cfg, k, b, 0.5, -0.1) == 0.0   # behind the element


# ------------------------------------------------------------------------- Eq. 11-16
@pytest.mark.parametrize("f,y,r,Rf", [(5e6, 0.0, 10e-3, 18e-3), (3e6, 0.0, 40e-3, 18e-3),
                                       (7e6, 0.8e-3, 15e-3, 18e-3), (5e6, -1.5e-3, 25e-3, 60e-3),
                                       (4e6, 0.5e-3, 30e-3, math.inf)])
def test_delta_is_gaussian_superposition_integral(oracle, f, y, r, Rf):
    cfg = _cfg(elev_focus=Rf).cfg
    h, k = cfg["height"], 2 * math.pi * f / cfg["c"]
    A, B = np.array([0.187 + 0.275j, 0.288 - 1.954j, 0.187 - 0.275j, 0.288 + 1.954j]), \
        np.array([4.558 - 25.59j, 8.598 - 7.924j, 4.558 + 25.59j, 8.598 + 7.924j])
    inv_rf = 0.0 if math.isinf(Rf) else 1 / Rf

    def integrand(yp):      # right-hand side of Eq. 11 with Pi replaced by Eq. 12
        pi_approx = (A * np.exp(-B * (yp / h) ** 2)).sum()
        return pi_approx * np.exp(-1j * k * yp**2 / 2 * inv_rf) * np.exp(1j * k * (y - yp) ** 2 / (2 * r))

    integ = quad_c(integrand, -3 * h, 3 * h, points=[-h / 2, 0, h / 2])
    assert oracle.delta(cfg, k, y, r) == pytest.approx(integ, rel=1e-7)

    def rect(yp):           # Eq. 11 itself (the exact elevation integral)
        return np.exp(-1j * k * yp**2 / 2 * inv_rf) * np.exp(1j * k * (y - yp) ** 2 / (2 * r))

    exact = quad_c(rect, -h / 2, h / 2)
    assert abs(oracle.delta(cfg, k, y, r) - exact) < 0.2 * abs(exact)


def test_delta_two_dimensional_limit(oracle):
    """Section V: h, R_f -> inf with G = 1, A = 1, B = 0 gives sqrt(2 i pi r / k); the
    four-Gaussian set gives (sum A_g) times that, sum A_g = 0.95."""
    cfg = _cfg(height=1e4, elev_focus=math.inf).cfg
    for f, r in ((3e6, 0.01), (6e6, 0.05)):
        k = 2 * math.pi * f / cfg["c"]
        want = 0.95 * np.sqrt(2j * math.pi * r / k)
        assert oracle.delta(cfg, k, 0.0, r) == pytest.approx(want, rel=1e-6)


def test_delta_small_height_limit(oracle):
    """h -> 0: alpha_g -> B_g / h^2, delta -> h sum_g A_g sqrt(pi / B_g) (real)."""
    cfg = _cfg(height=1e-6).cfg
    k = 2 * math.pi * 5e6 / 1540
    d = oracle.delta(cfg, k, 0.0, 0.02)
    A, B = oracle.gaussian_coefficients()
    lim = 1e-6 * (A * np.sqrt(np.pi / B)).sum()
    assert abs(lim.imag) < 1e-18
    assert d == pytest.approx(lim, rel=1e-4)
    assert lim.real == pytest.approx(0.99190e-6, rel=1e-4)


# ------------------------------------------------------------------------- Eq. 40
def test_attenuation_units(oracle):
    """One-way loss in dB is alpha [dB/cm/MHz] * f [MHz] * r [cm] * (20/ln10)/8.69."""
    w0 = _cfg(alpha_db=0.0).cfg
    w1 = dict(w0, alpha_db=0.7)
    f, Z = 6e6, 30e-3
    g0 = oracle.green(w0, f, 0.0, 0.0, Z, 0)
    g1 = oracle.green(w1, f, 0.0, 0.0, Z, 0)
    xc, _, _ = oracle.centroids(w0)
    r = math.hypot(xc[0], Z)
    loss_db = -20 * math.log10(abs(g1) / abs(g0))
    assert loss_db == pytest.approx(0.7 * 6 * (r * 100) * (20 / math.log(10)) / 8.69, rel=1e-10)
    assert loss_db == pytest.approx(0.7 * 6 * r * 100, rel=1e-3)
    assert np.angle(g1 / g0) == pytest.approx(0.0, abs=1e-12)


# -------------------------------------------------------------- Fig. 14-15, App. C
@pytest.mark.parametrize("baffle", [0, 1])
def test_subelement_sum_converges_to_aperture_integral(oracle, baffle):
    """One element of width 2b = 2 lambda split in nu far-field sub-elements converges to
    the aperture integral of e^{ikr'}/r' delta(Y, r', k) (obliquity) over x' as nu grows."""
    f, c = 5e6, 1540.0
    lam = c / f
    k = 2 * math.pi / lam
    errs = []
    for X, Y, Z in ((0.0, 0.0, 5 * lam), (2.5 * lam, 0.0, 4 * lam), (-1.0 * lam, 0.3e-3, 6 * lam)):
        cfg_base = dict(ph.linear_probe(1, f, 2 * lam, 0.0, baffle=baffle), **ph.medium(f, alpha_db=0.0),
                        n_samples=100)
        b = lam

        def integrand(xp):
            rho = math.hypot(X - xp, Z)
            r = math.sqrt(rho * rho + Y * Y)
            ob = Z / rho if baffle == 0 else 1.0
            return np.exp(1j * k * r) / r * oracle.delta(cfg_base, k, Y, r) * ob

        exact = quad_c(integrand, -b, b)
        e_nu = []
        for nu in (1, 2, 4, 8, 16, 32):
            cfg = dict(cfg_base, n_sub=nu)
            s = sum(oracle.green(cfg, f, X, Y, Z, n) for n in range(nu)) * (2 * b / nu)
            e_nu.append(abs(s - exact) / abs(exact))
        assert all(e_nu[i + 1] < e_nu[i] for i in range(len(e_nu) - 1)), e_nu
        assert e_nu[-1] < 2e-3
        errs.append(e_nu)


# ------------------------------------------------------------ Section V: the 2-D case
def test_two_d_green_is_the_three_d_limit(oracle):
    """Eq. 35-36: with h, R_f -> inf the 3-D term e^{ikr}/r D delta tends to
    0.95 sqrt(2 i pi / k) e^{ikr}/sqrt(r) D, i.e. (sum A_g) sqrt(2 i pi / k) times the
    2-D term (the 3-D delta itself is pinned by quadrature above)."""
    base = ph.tiny(n_elements=3, n_sub=2, height=1e4, elev_focus=math.inf).cfg
    c2 = dict(base, two_d=1)
    for f, X, Z, n in ((3e6, 0.4e-3, 7e-3, 0), (6e6, -1.5e-3, 11e-3, 3), (4.5e6, 2e-3, 5e-3, 5)):
        k = 2 * math.pi * f / base["c"]
        g3 = oracle.green(base, f, X, 0.0, Z, n)
        g2 = oracle.green(c2, f, X, 0.0, Z, n)
        assert abs(g2) > 0
        assert g3 == pytest.approx(0.95 * np.sqrt(2j * math.pi / k) * g2, rel=1e-6)


def test_two_d_is_independent_of_height_and_focus(oracle):
    a = ph.tiny(two_d=True, height=5e-3, elev_focus=18e-3).cfg
    b = dict(a, height=1e-2, elev_focus=math.inf)
    for f, X, Z, n in ((5e6, 0.3e-3, 6e-3, 1), (7e6, -0.9e-3, 10e-3, 2)):
        assert oracle.green(a, f, X, 0.0, Z, n) == oracle.green(b, f, X, 0.0, Z, n)


@pytest.mark.parametrize("baffle", [0, 1])
def test_two_d_subelement_sum_converges_to_line_aperture_integral(oracle, baffle):
    """Eq. 37 with one element: the nu far-field sub-elements (width 2b/nu each)
    converge to the integral of e^{ikr'}/sqrt(r') (obliquity) over the aperture."""
    f, c = 5e6, 1540.0
    lam = c / f
    k = 2 * math.pi / lam
    b = lam
    cfg_base = dict(ph.linear_probe(1, f, 2 * lam, 0.0, baffle=baffle), **ph.medium(f, alpha_db=0.0),
                    n_samples=100, two_d=1)
    for X, Z in ((0.0, 5 * lam), (2.5 * lam, 4 * lam), (-1.0 * lam, 6 * lam)):
        def integrand(xp):
            r = math.hypot(X - xp, Z)
            ob = Z / r if baffle == 0 else 1.0
            return np.exp(1j * k * r) / math.sqrt(r) * ob

        exact = quad_c(integrand, -b, b)
        e_nu = []
        for nu in (1, 2, 4, 8, 16, 32):
            cfg = dict(cfg_base, n_sub=nu)
            s = sum(oracle.green(cfg, f, X, 0.0, Z, n) for n in range(nu)) * (2 * b / nu)
            e_nu.append(abs(s - exact) / abs(exact))
        assert all(e_nu[i + 1] < e_nu[i] for i in range(len(e_nu) - 1)), e_nu
        assert e_nu[-1] < 2e-3


def test_two_d_two_way_arrival_time(oracle):
    """2-D (Eq. 38): one element transmits, one scatterer; the echo envelope on element m
    peaks at (r_tx + r_rx)/c."""
    w = ph.tiny(n_elements=4, n_sub=1, n_tx=1, alpha_db=0.0, nt=1200, two_d=True)
    cfg = w.cfg
    delays = np.zeros((1, 4))
    apod = np.zeros((1, 4))
    apod[0, 2] = 1.0
    X, Z = np.array([-0.4e-3]), np.array([8e-3])
    lo, hi, n = oracle.bins(cfg)
    q = np.arange(lo, hi + 1)
    Xq = oracle.rf_spectrum(cfg, delays, apod, X, None, Z, [1.0], q)[0]
    xc, _, _ = oracle.centroids(cfg)
    c, fs, nt = cfg["c"], cfg["fs"], cfg["n_samples"]
    wq = 2 * np.pi * q * fs / nt
    for m in range(4):
        tau = (math.hypot(X[0] - xc[2], Z[0]) + math.hypot(X[0] - xc[m], Z[0])) / c
        t = tau + np.linspace(-2, 2, 4001) / fs
        env = np.abs(np.exp(-1j * np.outer(t, wq)) @ Xq[m])
        assert abs(t[np.argmax(env)] - tau) * fs < 2e-3


# ------------------------------------------------------------------- arrival time
@pytest.mark.parametrize("delay_us", [0.0, 2.0])
def test_two_way_arrival_time(oracle, delay_us):
    """One element transmits (delay dtau), one scatterer: the envelope of the echo on
    element m peaks at (r_tx + r_rx)/c + dtau.  h = 10 um makes delta real and flat."""
    w = ph.tiny(n_elements=4, n_sub=1, n_tx=1, height=10e-6, alpha_db=0.0, nt=1200)
    cfg = w.cfg
    delays = np.zeros((1, 4))
    delays[0, 1] = delay_us * 1e-6
    apod = np.zeros((1, 4))
    apod[0, 1] = 1.0
    X, Z = np.array([0.6e-3]), np.array([9e-3])
    lo, hi, n = oracle.bins(cfg)
    q = np.arange(lo, hi + 1)
    Xq = oracle.rf_spectrum(cfg, delays, apod, X, None, Z, [1.0], q)[0]     # [N][nq]
    xc, _, _ = oracle.centroids(cfg)
    c, fs, nt = cfg["c"], cfg["fs"], cfg["n_samples"]
    wq = 2 * np.pi * q * fs / nt
    for m in range(4):
        tau = (math.hypot(X[0] - xc[1], Z[0]) + math.hypot(X[0] - xc[m], Z[0])) / c + delays[0, 1]
        t = tau + np.linspace(-2, 2, 4001) / fs
        env = np.abs(np.exp(-1j * np.outer(t, wq)) @ Xq[m])
        assert abs(t[np.argmax(env)] - tau) * fs < 2e-3
    # and in the time signals: peak of the analytic envelope within one sample
    rf = oracle.rf(cfg, delays, apod, X, None, Z, [1.0])[0]
    spec = np.fft.fft(rf, axis=-1)
    spec[:, nt // 2 + 1:] = 0
    spec[:, 1:nt // 2] *= 2
    env = np.abs(np.fft.ifft(spec, axis=-1))
    for m in range(4):
        tau = (math.hypot(X[0] - xc[1], Z[0]) + math.hypot(X[0] - xc[m], Z[0])) / c + delays[0, 1]
        assert abs(np.argmax(env[m]) - tau * fs) <= 1.0


# --------------------------------------------------------------- Eq. 29-33 invariants
def test_reciprocity(oracle):
    """Single-element transmits: echo of transmit i on element j equals that of j on i."""
    w = ph.tiny(n_elements=5, n_sub=2, n_scat=6, convex=False)
    N = 5
    delays, apod = np.zeros((N, N)), np.eye(N)
    lo, hi, _ = oracle.bins(w.cfg)
    q = [lo, (lo + hi) // 2, hi]
    X = oracle.rf_spectrum(w.cfg, delays, apod, w.x, None, w.z, w.rc, q)     # [t][e][q]
    np.testing.assert_allclose(X, np.transpose(X, (1, 0, 2)), rtol=1e-12, atol=1e-14 * np.abs(X).max())
    assert np.abs(X - np.transpose(X, (1, 0, 2))).max() < 1e-12 * np.abs(X).max()


def test_linearity_and_superposition(oracle):
    w = ph.tiny(n_elements=4, n_sub=2, n_scat=8, n_tx=2, y_spread=1e-3)
    args = (w.cfg, w.delays, w.apod)
    r2 = ph.normal(99, 1, 8)
    full = oracle.rf(*args, w.x, w.y, w.z, w.rc.astype(np.float64) + 2.0 * r2)
    a = oracle.rf(*args, w.x, w.y, w.z, w.rc)
    b = oracle.rf(*args, w.x, w.y, w.z, r2)
    np.testing.assert_allclose(full, a + 2 * b, atol=1e-11 * np.abs(full).max())
    part1 = oracle.rf(*args, w.x[:3], w.y[:3], w.z[:3], w.rc[:3])
    part2 = oracle.rf(*args, w.x[3:], w.y[3:], w.z[3:], w.rc[3:])
    np.testing.assert_allclose(a, part1 + part2, atol=1e-11 * np.abs(a).max())


def test_subelement_sum_equals_finer_probe(oracle):
    """Eq. 24 + Eq. 33: with kerf 0, an N-element probe split in nu = 2 is a 2N-element
    probe of half pitch whose element pairs share delay and apodisation; the element
    echo is the sum of the pair's echoes."""
    N, p, f = 4, 0.3e-3, 5e6
    med = ph.medium(f)
    A = dict(ph.linear_probe(N, f, p, 0.0, n_sub=2), **med, n_samples=400)
    B = dict(ph.linear_probe(2 * N, f, p / 2, 0.0, n_sub=1), **med, n_samples=400)
    w = ph.tiny(n_elements=N, n_scat=5, n_tx=2)
    dA, aA = w.delays.astype(np.float64), w.apod.astype(np.float64)
    dB, aB = np.repeat(dA, 2, axis=1), np.repeat(aA, 2, axis=1)
    lo, hi, _ = oracle.bins(A)
    q = [lo, lo + 7, (lo + hi) // 2, hi]
    XA = oracle.rf_spectrum(A, dA, aA, w.x, None, w.z, w.rc, q)
    XB = oracle.rf_spectrum(B, dB, aB, w.x, None, w.z, w.rc, q)
    np.testing.assert_allclose(XA, XB[:, 0::2] + XB[:, 1::2], rtol=1e-10,
                               atol=1e-12 * np.abs(XA).max())


# -------------------------------------------------------------------------- R5 iDFT
def test_idft_is_numpy_fft(oracle):
    rng = np.random.default_rng(0)
    nt = 250
    q = np.arange(17, 93)
    X = rng.normal(size=(3, len(q))) + 1j * rng.normal(size=(3, len(q)))
    full = np.zeros((3, nt), complex)
    full[:, q] = X
    np.testing.assert_allclose(oracle.idft(X, q, nt), np.fft.fft(full, axis=-1).real,
                               atol=1e-12)


# -------------------------------------------------------------------------- Eq. 41-42
def test_pfield_midpoint_sum_approximates_integral(oracle):
    w = ph.tiny(n_elements=3, n_sub=1, n_tx=1)
    cfg = w.cfg
    X, Y, Z = 0.4e-3, 0.0, 8e-3
    xc, _, _ = oracle.centroids(cfg)
    wc = 2 * np.pi * cfg["fc"]
    ws = np.linspace(1e-3 * wc, 2 * wc, 6001)

    def P(wv):
        f = wv / (2 * np.pi)
        tot = 0j
        for n in range(3):
            tot += w.apod[0, n] * oracle.green(cfg, f, X, Y, Z, n) * np.exp(1j * wv * w.delays[0, n])
        return tot * oracle.pulse_spectrum(cfg, wv)[0] * math.sqrt(oracle.transducer_response(cfg, wv)[0])

    ref = math.sqrt(integrate.trapezoid([abs(P(v)) ** 2 for v in ws], ws))
    r_max = max(math.hypot(X - x, Z) for x in xc)
    nf = oracle.pfield_nfreq(cfg, r_max, float(w.delays.max()))
    assert nf == math.ceil(2 * wc / (2 * np.pi / (r_max / cfg["c"] + float(w.delays.max()))))
    for mult, tol in ((1, 0.05), (8, 2e-4)):
        prms = oracle.pfield(cfg, w.delays, w.apod, [X], [Y], [Z], mult * nf)[0, 0]
        assert prms == pytest.approx(ref, rel=tol)


# -------------------------------------------------------------------- gradients (FD)
@pytest.mark.parametrize("convex,y,two_d", [(False, 0.0, False), (True, 0.0, False),
                                            (False, 0.7e-3, False), (True, 0.0, True)])
def test_green_grad_finite_differences(oracle, convex, y, two_d):
    cfg = ph.tiny(convex=convex, n_sub=2, two_d=two_d).cfg
    h = 1e-8
    for (X, Z, n, f) in ((0.5e-3, 6e-3, 1, 4e6), (-1.2e-3, 9e-3, 3, 6.5e6)):
        g, gx, gz = oracle.green_grad(cfg, f, X, y, Z, n)
        assert g == pytest.approx(oracle.green(cfg, f, X, y, Z, n), rel=1e-14)
        fx = (oracle.green(cfg, f, X + h, y, Z, n) - oracle.green(cfg, f, X - h, y, Z, n)) / (2 * h)
        fz = (oracle.green(cfg, f, X, y, Z + h, n) - oracle.green(cfg, f, X, y, Z - h, n)) / (2 * h)
        assert gx == pytest.approx(fx, rel=2e-6)
        assert gz == pytest.approx(fz, rel=2e-6)


@pytest.mark.parametrize("two_d", [False, True])
def test_rf_grad_finite_differences(oracle, two_d):
    w = ph.tiny(n_elements=4, n_sub=2, n_scat=4, n_tx=2, nt=256, two_d=two_d)
    cfg = w.cfg
    x, z, R = (w.x.astype(np.float64), w.z.astype(np.float64), w.rc.astype(np.float64))
    d, a = w.delays.astype(np.float64), w.apod.astype(np.float64)
    tgt = oracle.rf(cfg, d, a, x + 2e-5, None, z - 1e-5, 0.9 * R)

    def loss(x_, z_, R_, d_):
        r = oracle.rf(cfg, d_, a, x_, None, z_, R_)
        return float(((r - tgt) ** 2).sum()), r

    L0, r0 = loss(x, z, R, d)
    gR, gx, gz, gd = oracle.rf_grad(cfg, d, a, x, None, z, R, 2 * (r0 - tgt))
    hp, hr, ht = 1e-9, 1e-7, 1e-12
    for s in range(len(x)):
        e = np.zeros_like(x)
        e[s] = 1
        fdR = (loss(x, z, R + hr * e, d)[0] - loss(x, z, R - hr * e, d)[0]) / (2 * hr)
        fdx = (loss(x + hp * e, z, R, d)[0] - loss(x - hp * e, z, R, d)[0]) / (2 * hp)
        fdz = (loss(x, z + hp * e, R, d)[0] - loss(x, z - hp * e, R, d)[0]) / (2 * hp)
        assert gR[s] == pytest.approx(fdR, rel=1e-6)
        assert gx[s] == pytest.approx(fdx, rel=1e-6)
        assert gz[s] == pytest.approx(fdz, rel=1e-6)
    for t, e_ in ((0, 0), (1, 2), (0, 3)):
        E = np.zeros_like(d)
        E[t, e_] = 1
        fdd = (loss(x, z, R, d + ht * E)[0] - loss(x, z, R, d - ht * E)[0]) / (2 * ht)
        assert gd[t, e_] == pytest.approx(fdd, rel=1e-6)
