"""Seeded synthetic inputs: probes, media, transmit sequences and speckle phantoms.

This module holds no arithmetic of the simulation model itself.  It produces the
*inputs* the model is applied to, in the float32 form a caller hands the library:
scatterer positions and reflection coefficients, and per-element transmit delays and
apodisation (the delay laws below use element centres only; they are the caller's
choice, not part of the paper's equations).  Both the CUDA path and the FP64 oracle
receive exactly these arrays.

Random numbers come from a counter-based generator written out here (SplitMix64 of
(seed, stream, index), Box-Muller for normals), so the same seed gives the same
phantom on every machine and numpy version.

The synthetic workloads stand in for the paper's phantoms (B-mode phantom of 39,500
scatterers, Section VIII-A; Doppler phantom of ~26,000 scatterers, Section VIII-B),
which are not available: uniform speckle with N(0, 1) reflection coefficients.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """SplitMix64 output for counters (seed, stream, 0..n-1)."""
    base = np.uint64((seed * 0x100000001B3 + stream * 0xC2B2AE3D27D4EB4F) & (2**64 - 1))
    with np.errstate(over="ignore"):
        z = base + (np.arange(1, n + 1, dtype=np.uint64) * _GAMMA)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles uniform in [0, 1)."""
    return (_splitmix64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * 2.0**-53


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller."""
    u1 = 1.0 - uniform(seed, stream, n)          # (0, 1]
    u2 = uniform(seed, stream + 1_000_003, n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------- probes
def linear_probe(n_elements, fc, pitch, kerf, height=5e-3, elev_focus=18e-3, n_sub=0,
                 frac_bw=0.75, baffle=0, zeta=1.75):
    return dict(n_elements=int(n_elements), pitch=float(pitch), width=float(pitch - kerf),
                height=float(height), elev_focus=float(elev_focus), radius=0.0,
                fc=float(fc), frac_bw=float(frac_bw), n_sub=int(n_sub), baffle=int(baffle),
                zeta=float(zeta))


def convex_probe(n_elements, fc, pitch, kerf, radius, height=5e-3, elev_focus=60e-3,
                 n_sub=0, frac_bw=0.75, baffle=0, zeta=1.75):
    d = linear_probe(n_elements, fc, pitch, kerf, height, elev_focus, n_sub, frac_bw,
                     baffle, zeta)
    d["radius"] = float(radius)
    return d


def medium(fc, c=1540.0, alpha_db=0.5, fs_factor=4.0, pulse=0, pulse_cycles=1.0):
    return dict(c=float(c), alpha_db=float(alpha_db), fs=float(fs_factor * fc),
                pulse=int(pulse), pulse_cycles=float(pulse_cycles))


def element_centres(probe) -> tuple[np.ndarray, np.ndarray]:
    """Element centres (x, z) used by the delay laws (linear: z = 0; convex: on the arc
    of radius R about (0, -R), spaced by the pitch along the arc)."""
    N, p = probe["n_elements"], probe["pitch"]
    k = np.arange(N) - (N - 1) / 2.0
    if probe["radius"] > 0:
        R = probe["radius"]
        a = k * p / R
        return R * np.sin(a), R * np.cos(a) - R
    return k * p, np.zeros(N)


# ------------------------------------------------------------------------- delay laws
def focused_delays(probe, c, focus_x, focus_z):
    """Delays that make all element wavefronts meet at (focus_x, focus_z)."""
    xe, ze = element_centres(probe)
    d = np.hypot(xe - focus_x, ze - focus_z)
    return ((d.max() - d) / c)[None, :]


def plane_wave_delays(probe, c, angles_rad):
    xe, _ = element_centres(probe)
    out = []
    for a in np.atleast_1d(angles_rad):
        t = xe * math.sin(a) / c
        out.append(t - t.min())
    return np.array(out)


def diverging_delays(probe, c, angles_rad):
    """Diverging waves from virtual sources at half the radius behind the convex
    surface, along each angle from the centre of curvature."""
    xe, ze = element_centres(probe)
    R = probe["radius"]
    out = []
    for a in np.atleast_1d(angles_rad):
        vx, vz = 0.5 * R * math.sin(a), -R + 0.5 * R * math.cos(a)
        d = np.hypot(xe - vx, ze - vz)
        out.append((d - d.min()) / c)
    return np.array(out)


# -------------------------------------------------------------------------- workloads
@dataclass
class Workload:
    """One simulation problem: plain-number description plus float32 arrays."""
    name: str
    cfg: dict                 # probe + medium + n_samples
    delays: np.ndarray        # [T][N] float32, seconds
    apod: np.ndarray          # [T][N] float32
    x: np.ndarray             # [S] float32, metres
    y: np.ndarray | None      # [S] float32 or None (Y = 0)
    z: np.ndarray             # [S] float32
    rc: np.ndarray            # [S] float32 reflection coefficients
    extra: dict = field(default_factory=dict)

    @property
    def n_tx(self):
        return self.delays.shape[0]

    @property
    def n_scat(self):
        return len(self.x)


def rf_length(cfg, x, z, delays, y=None) -> int:
    """An even RF length covering the farthest two-way path plus the pulse tails:
    Nt >= fs (2 r_max / c + max delay + 8 / fc), r_max over element edges."""
    xe, ze = element_centres(cfg)
    half = cfg["width"] / 2.0
    y2 = 0.0 if y is None else float(np.max(np.asarray(y, np.float64) ** 2))
    xs, zs = np.asarray(x, np.float64), np.asarray(z, np.float64)
    if cfg["radius"] <= 0:
        # linear array: (x - x_e)^2 is convex in x_e, so the farthest edge is an end one
        xe, ze = np.array([xe.min(), xe.max()]), np.zeros(2)
    r2 = 0.0
    for s0 in range(0, len(xs), 1 << 16):
        xc, zc = xs[s0:s0 + (1 << 16)], zs[s0:s0 + (1 << 16)]
        for sgn in (-1.0, 1.0):
            dx = xc[:, None] - (xe[None, :] + sgn * half)
            dz = zc[:, None] - ze[None, :]
            r2 = max(r2, float(np.max(dx * dx + dz * dz)))
    r_max = math.sqrt(r2 + y2)
    t = 2.0 * r_max / cfg["c"] + float(np.max(delays)) + 8.0 / cfg["fc"]
    n = int(math.ceil(cfg["fs"] * t))
    return n + (n & 1)


def _box(seed, S, x0, x1, z0, z1):
    x = x0 + (x1 - x0) * uniform(seed, 1, S)
    z = z0 + (z1 - z0) * uniform(seed, 2, S)
    rc = normal(seed, 3, S)
    return x, z, rc


def _finish(name, probe, med, delays, x, z, rc, y=None, apod=None, nt=None, **extra):
    cfg = dict(probe)
    cfg.update(med)
    delays = np.asarray(delays, np.float32)
    apod = np.ones_like(delays) if apod is None else np.asarray(apod, np.float32)
    x, z, rc = (np.asarray(a, np.float32) for a in (x, z, rc))
    y = None if y is None else np.asarray(y, np.float32)
    cfg["n_samples"] = int(nt) if nt else rf_length(cfg, x, z, delays, y)
    return Workload(name, cfg, delays, apod, x, y, z, rc, dict(extra))


def focused_linear_64(seed=1001, n_scat=200):
    """64-element 5 MHz linear array, one focused transmit at (0, 20 mm), 1-cycle Hann
    pulse, 200 scatterers in x in [-10, 10] mm, z in [5, 35] mm."""
    probe = linear_probe(64, 5e6, 0.30e-3, 0.03e-3, n_sub=2)
    med = medium(5e6, pulse=1)
    x, z, rc = _box(seed, n_scat, -10e-3, 10e-3, 5e-3, 35e-3)
    return _finish("focused-linear-64 (5 MHz, 200 scatterers)", probe, med,
                   focused_delays(probe, med["c"], 0.0, 20e-3), x, z, rc)


def planewave_linear_128(seed=1002, n_scat=20000, with_points=True):
    """128-element 7.6 MHz linear array, nu = 3, one 0-degree plane wave, speckle in a
    38 x 40 mm box from z = 5 mm plus three bright points at z = 10/20/30 mm."""
    probe = linear_probe(128, 7.6e6, 0.30e-3, 0.03e-3, n_sub=3)
    med = medium(7.6e6)
    x, z, rc = _box(seed, n_scat, -19e-3, 19e-3, 5e-3, 45e-3)
    if with_points:
        x = np.concatenate([x, [0.0, 0.0, 0.0]])
        z = np.concatenate([z, [10e-3, 20e-3, 30e-3]])
        rc = np.concatenate([rc, [10.0, 10.0, 10.0]])
    return _finish(f"planewave-linear-128 (7.6 MHz, nu 3, {len(x)} scatterers)", probe, med,
                   plane_wave_delays(probe, med["c"], [0.0]), x, z, rc)


def planewave_linear_128_2d(seed=1002, n_scat=20000, with_points=True):
    """The planewave-linear-128 problem in the 2-D x-z model of Section V (Eq. 36-38)."""
    w = planewave_linear_128(seed, n_scat, with_points)
    w.cfg["two_d"] = 1
    w.name = w.name.replace("planewave-linear-128", "planewave-linear-128-2d")
    return w


def diverging_convex_128_3d(seed=1003, n_scat=100000, n_tx=31, y_half=2.5e-3):
    """The diverging-convex-128 problem with a 3-D scatterer cloud: elevations uniform in
    [-y_half, y_half] (the element height is 5 mm), so that delta carries the Eq. 14
    exponent (beta, gamma != 0; Section VIII's 3-D case)."""
    w = diverging_convex_128(seed, n_scat, n_tx)
    w.y = (y_half * (2.0 * uniform(seed, 9, w.n_scat) - 1.0)).astype(np.float32)
    w.cfg["n_samples"] = rf_length(w.cfg, w.x, w.z, w.delays, w.y)
    w.name = w.name.replace("diverging-convex-128", "diverging-convex-128-3d")
    return w


def pfield_l11_5v(nx=201, nz=201, tilt_deg=10.0):
    """Fig. 10 setup for the RMS field (Eq. 41-42): 128-element 7.6 MHz linear array,
    pitch 0.27 mm, kerf 30 um, 77 % bandwidth, elevation focus 18 mm, one plane wave tilted
    by tilt_deg; an nx x nz grid over x in [-20, 20] mm, z in [0.5, 40] mm at y = 0."""
    probe = linear_probe(128, 7.6e6, 0.27e-3, 0.03e-3, elev_focus=0.018, frac_bw=0.77)
    med = medium(7.6e6)
    X, Z = np.meshgrid(np.linspace(-20e-3, 20e-3, nx), np.linspace(0.5e-3, 40e-3, nz))
    delays = plane_wave_delays(probe, med["c"], [math.radians(tilt_deg)])
    cfg = dict(probe)
    cfg.update(med)
    cfg["n_samples"] = 64   # unused by the field; a plan needs one
    return Workload("pfield-l11-5v", cfg, np.asarray(delays, np.float32),
                    np.ones_like(delays, dtype=np.float32), X.ravel().astype(np.float32), None,
                    Z.ravel().astype(np.float32), np.zeros(X.size, np.float32),
                    dict(nx=nx, nz=nz))


def diverging_convex_128(seed=1003, n_scat=100000, n_tx=31):
    """128-element 3 MHz convex array (R = 60 mm, pitch 0.5 mm, nu = 2), 31 diverging
    waves over +-20 degrees, speckle uniform in area in a 60-degree sector to 120 mm."""
    R = 60e-3
    probe = convex_probe(128, 3e6, 0.50e-3, 0.05e-3, R, n_sub=2)
    med = medium(3e6)
    ang = np.deg2rad(-30 + 60 * uniform(seed, 1, n_scat))
    rad = np.sqrt(R**2 + ((R + 120e-3) ** 2 - R**2) * uniform(seed, 2, n_scat))
    x, z = rad * np.sin(ang), rad * np.cos(ang) - R
    rc = normal(seed, 3, n_scat)
    return _finish(f"diverging-convex-128 (3 MHz, {n_tx} tx, {n_scat} scatterers)", probe, med,
                   diverging_delays(probe, med["c"], np.deg2rad(np.linspace(-20, 20, n_tx))),
                   x, z, rc)


def planewave_linear_128_grad(seed=1004, n_scat=10000, n_tx=11):
    """128-element 5 MHz linear array (nu from Eq. 21), 11 plane waves over -10..10
    degrees; a target phantom from positions perturbed by N(0, 0.05 mm)."""
    probe = linear_probe(128, 5e6, 0.30e-3, 0.03e-3)
    med = medium(5e6)
    half = 128 * 0.30e-3 / 2
    x, z, rc = _box(seed, n_scat, -half, half, 5e-3, 45e-3)
    xt = x + 0.05e-3 * normal(seed, 11, n_scat)
    zt = z + 0.05e-3 * normal(seed, 13, n_scat)
    w = _finish(f"planewave-linear-128-grad (5 MHz, {n_tx} tx, {n_scat} scatterers)", probe, med,
                plane_wave_delays(probe, med["c"], np.deg2rad(np.linspace(-10, 10, n_tx))),
                x, z, rc)
    w.extra["x_target"] = np.asarray(xt, np.float32)
    w.extra["z_target"] = np.asarray(zt, np.float32)
    return w


def ragged_batch(seed=1005, n_sims=256, s_min=1000, s_max=1_000_000, scale=1.0):
    """Independent simulations of uneven size: N ~ U{64..192} linear 0.3 mm pitch,
    fc ~ U[3, 8] MHz, S log-uniform in [s_min, s_max] (times scale), T ~ U{1..75}
    plane waves over +-15 degrees."""
    sims = []
    uN = uniform(seed, 1, n_sims)
    ufc = uniform(seed, 2, n_sims)
    uS = uniform(seed, 3, n_sims)
    uT = uniform(seed, 4, n_sims)
    for i in range(n_sims):
        N = 64 + int(uN[i] * 129)
        fc = 3e6 + 5e6 * ufc[i]
        S = max(1, int(scale * math.floor(10 ** (math.log10(s_min)
                                                   + uS[i] * math.log10(s_max / s_min)))))
        T = 1 + int(uT[i] * 75)
        probe = linear_probe(N, fc, 0.30e-3, 0.03e-3)
        med = medium(fc)
        half = N * 0.30e-3 / 2
        x, z, rc = _box(seed * 1000 + i, S, -half, half, 5e-3, 45e-3)
        ang = np.deg2rad(np.linspace(-15, 15, T)) if T > 1 else np.array([0.0])
        sims.append(_finish(f"ragged[{i}]", probe, med,
                            plane_wave_delays(probe, med["c"], ang), x, z, rc))
    return sims


def tiny(seed=7, n_elements=4, n_scat=5, n_tx=2, n_sub=2, fc=5e6, nt=None, convex=False,
         baffle=0, pulse=0, y_spread=0.0, alpha_db=0.5, height=5e-3, elev_focus=18e-3,
         two_d=False):
    """Small problems for exhaustive checks (two_d: the 2-D model of Section V)."""
    if convex:
        probe = convex_probe(n_elements, fc, 0.5e-3, 0.05e-3, 20e-3, height=height,
                             elev_focus=elev_focus, n_sub=n_sub, baffle=baffle)
    else:
        probe = linear_probe(n_elements, fc, 0.3e-3, 0.03e-3, height=height,
                             elev_focus=elev_focus, n_sub=n_sub, baffle=baffle)
    if two_d:
        probe["two_d"] = 1
    med = medium(fc, pulse=pulse, alpha_db=alpha_db)
    x, z, rc = _box(seed, n_scat, -3e-3, 3e-3, 4e-3, 12e-3)
    y = None if y_spread == 0 else y_spread * (2 * uniform(seed, 5, n_scat) - 1)
    ang = np.deg2rad(np.linspace(-8, 8, n_tx)) if n_tx > 1 else np.array([3.0 * np.pi / 180])
    delays = plane_wave_delays(probe, med["c"], ang)
    apod = 0.5 + uniform(seed, 6, delays.size).reshape(delays.shape)
    return _finish("tiny", probe, med, delays, x, z, rc, y=y, apod=apod, nt=nt)
