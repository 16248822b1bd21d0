"""ctypes front end of the FP64 CPU oracle (``simus_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path never imports it,
and this module imports nothing from the CUDA package.

A problem is described by a plain dict (the vocabulary of ``phantoms``): probe
(n_elements, pitch, width, height, elev_focus, radius, fc, frac_bw, n_sub, baffle, zeta),
medium (c, alpha_db, fs, pulse, pulse_cycles) and n_samples.  Arrays are promoted to
float64 before they reach the C code.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simus_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (FP64, OpenMP, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("n_elements", C.c_int32), ("n_sub", C.c_int32), ("baffle", C.c_int32),
        ("pulse", C.c_int32), ("n_samples", C.c_int32), ("two_d", C.c_int32),
        ("pitch", C.c_double), ("width", C.c_double), ("height", C.c_double),
        ("elev_focus", C.c_double), ("radius", C.c_double), ("fc", C.c_double),
        ("frac_bw", C.c_double), ("zeta", C.c_double), ("c", C.c_double),
        ("alpha_db", C.c_double), ("fs", C.c_double), ("pulse_cycles", C.c_double),
    ]


_lib = None
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_P = C.POINTER(Params)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.oracle_transducer_response.restype = C.c_double
        L.oracle_transducer_response.argtypes = [_P, C.c_double]
        L.oracle_pulse_spectrum.argtypes = [_P, C.c_double, _D, _D]
        L.oracle_transfer.argtypes = [_P, C.c_double, _D, _D]
        L.oracle_nsub.restype = C.c_int32
        L.oracle_nsub.argtypes = [_P]
        L.oracle_bins.restype = C.c_int32
        L.oracle_bins.argtypes = [_P, _I32, _I32]
        L.oracle_centroids.argtypes = [_P, _D, _D, _D]
        L.oracle_delta.argtypes = [_P, C.c_double, C.c_double, C.c_double, _D, _D]
        L.oracle_directivity.restype = C.c_double
        L.oracle_directivity.argtypes = [_P, C.c_double, C.c_double, C.c_double, C.c_double]
        L.oracle_green.argtypes = [_P, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_int32, _D, _D]
        L.oracle_green_grad.argtypes = [_P, C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_int32, _D]
        L.oracle_rf_spectrum.argtypes = [_P, C.c_int32, _D, _D, C.c_int64, _D, _D, _D, _D,
                                         C.c_int32, _I32, _D]
        L.oracle_idft.argtypes = [C.c_int32, C.c_int32, C.c_int32, _I32, _D, _D]
        L.oracle_rf.restype = C.c_int32
        L.oracle_rf.argtypes = [_P, C.c_int32, _D, _D, C.c_int64, _D, _D, _D, _D, _D]
        L.oracle_pfield_nfreq.restype = C.c_int32
        L.oracle_pfield_nfreq.argtypes = [_P, C.c_double, C.c_double]
        L.oracle_pfield.argtypes = [_P, C.c_int32, _D, _D, C.c_int64, _D, _D, _D,
                                    C.c_int32, _D]
        L.oracle_rf_grad.argtypes = [_P, C.c_int32, _D, _D, C.c_int64, _D, _D, _D, _D, _D,
                                     _D, _D, _D, _D]
        L.oracle_gaussian_coefficients.argtypes = [_D, _D, _D, _D]
    return _lib


def params(cfg: dict) -> Params:
    p = Params()
    for name in ("n_elements", "n_sub", "baffle", "pulse", "n_samples", "two_d"):
        setattr(p, name, int(cfg.get(name, 0)))
    for name in ("pitch", "width", "height", "elev_focus", "radius", "fc", "frac_bw",
                 "zeta", "c", "alpha_db", "fs", "pulse_cycles"):
        setattr(p, name, float(cfg.get(name, 0.0)))
    return p


def _d(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a, a.ctypes.data_as(_D)


def _opt(a):
    if a is None:
        return None, None
    return _d(a)


# ---------------------------------------------------------------------------- spectra
def transducer_response(cfg, w):
    p = params(cfg)
    return np.array([lib().oracle_transducer_response(C.byref(p), float(x))
                     for x in np.atleast_1d(w)])


def _complex_fn(fn, cfg, w):
    p = params(cfg)
    out = []
    re, im = C.c_double(), C.c_double()
    for x in np.atleast_1d(w):
        fn(C.byref(p), float(x), C.byref(re), C.byref(im))
        out.append(re.value + 1j * im.value)
    return np.array(out)


def pulse_spectrum(cfg, w):
    return _complex_fn(lib().oracle_pulse_spectrum, cfg, w)


def transfer(cfg, w):
    return _complex_fn(lib().oracle_transfer, cfg, w)


def nsub(cfg) -> int:
    return int(lib().oracle_nsub(C.byref(params(cfg))))


def bins(cfg):
    lo, hi = C.c_int32(), C.c_int32()
    n = lib().oracle_bins(C.byref(params(cfg)), C.byref(lo), C.byref(hi))
    return int(lo.value), int(hi.value), int(n)


def gaussian_coefficients():
    a = [np.zeros(4) for _ in range(4)]
    lib().oracle_gaussian_coefficients(*[x.ctypes.data_as(_D) for x in a])
    return a[0] + 1j * a[1], a[2] + 1j * a[3]


# --------------------------------------------------------------------------- geometry
def centroids(cfg):
    m = nsub(cfg) * int(cfg["n_elements"])
    xc, zc, psi = np.zeros(m), np.zeros(m), np.zeros(m)
    lib().oracle_centroids(C.byref(params(cfg)), xc.ctypes.data_as(_D),
                           zc.ctypes.data_as(_D), psi.ctypes.data_as(_D))
    return xc, zc, psi


def delta(cfg, k, y, r) -> complex:
    re, im = C.c_double(), C.c_double()
    lib().oracle_delta(C.byref(params(cfg)), float(k), float(y), float(r),
                       C.byref(re), C.byref(im))
    return re.value + 1j * im.value


def directivity(cfg, k, bh, sin_t, cos_t) -> float:
    return float(lib().oracle_directivity(C.byref(params(cfg)), float(k), float(bh),
                                          float(sin_t), float(cos_t)))


def green(cfg, f, X, Y, Z, n) -> complex:
    re, im = C.c_double(), C.c_double()
    lib().oracle_green(C.byref(params(cfg)), float(f), float(X), float(Y), float(Z), int(n),
                       C.byref(re), C.byref(im))
    return re.value + 1j * im.value


def green_grad(cfg, f, X, Y, Z, n):
    out = np.zeros(6)
    lib().oracle_green_grad(C.byref(params(cfg)), float(f), float(X), float(Y), float(Z),
                            int(n), out.ctypes.data_as(_D))
    return out[0] + 1j * out[1], out[2] + 1j * out[3], out[4] + 1j * out[5]


# ------------------------------------------------------------------------------- RF
def rf_spectrum(cfg, delays, apod, x, y, z, rc, qlist):
    """X_q(e, t) at the listed bins, shape [T][N][len(qlist)] complex128."""
    delays, dp = _d(delays)
    apod, ap = _d(apod)
    T, N = delays.shape
    x, xp = _d(x)
    y, yp = _opt(y)
    z, zp = _d(z)
    rc, rp = _d(rc)
    q = np.ascontiguousarray(np.asarray(qlist, dtype=np.int32))
    out = np.zeros((T, N, len(q), 2))
    lib().oracle_rf_spectrum(C.byref(params(cfg)), T, dp, ap, len(x), xp, yp, zp, rp,
                             len(q), q.ctypes.data_as(_I32), out.ctypes.data_as(_D))
    return out[..., 0] + 1j * out[..., 1]


def idft(X, qlist, nt):
    """Direct inverse DFT of R5 over the last axis of X (complex, [..., nq])."""
    X = np.asarray(X, dtype=np.complex128)
    shape = X.shape[:-1]
    nq = X.shape[-1]
    Xi = np.ascontiguousarray(np.stack([X.real, X.imag], -1).reshape(-1, nq, 2))
    q = np.ascontiguousarray(np.asarray(qlist, dtype=np.int32))
    rf = np.zeros((Xi.shape[0], nt))
    lib().oracle_idft(Xi.shape[0], int(nt), nq, q.ctypes.data_as(_I32),
                      Xi.ctypes.data_as(_D), rf.ctypes.data_as(_D))
    return rf.reshape(shape + (nt,))


def rf(cfg, delays, apod, x, y, z, rc):
    """RF time signals [T][N][Nt] (float64)."""
    delays, dp = _d(delays)
    apod, ap = _d(apod)
    T, N = delays.shape
    x, xp = _d(x)
    y, yp = _opt(y)
    z, zp = _d(z)
    rc, rp = _d(rc)
    out = np.zeros((T, N, int(cfg["n_samples"])))
    lib().oracle_rf(C.byref(params(cfg)), T, dp, ap, len(x), xp, yp, zp, rp,
                    out.ctypes.data_as(_D))
    return out


def rf_grad(cfg, delays, apod, x, y, z, rc, drf):
    """Gradients (dL/dR, dL/dX, dL/dZ, dL/d delays) for the upstream gradient drf."""
    delays, dp = _d(delays)
    apod, ap = _d(apod)
    T, N = delays.shape
    x, xp = _d(x)
    y, yp = _opt(y)
    z, zp = _d(z)
    rc, rp = _d(rc)
    drf, gp = _d(drf)
    S = len(x)
    gR, gx, gz, gd = np.zeros(S), np.zeros(S), np.zeros(S), np.zeros((T, N))
    lib().oracle_rf_grad(C.byref(params(cfg)), T, dp, ap, S, xp, yp, zp, rp, gp,
                         gR.ctypes.data_as(_D), gx.ctypes.data_as(_D),
                         gz.ctypes.data_as(_D), gd.ctypes.data_as(_D))
    return gR, gx, gz, gd


# ----------------------------------------------------------------------------- pfield
def pfield_nfreq(cfg, r_max, tau_max) -> int:
    return int(lib().oracle_pfield_nfreq(C.byref(params(cfg)), float(r_max), float(tau_max)))


def pfield(cfg, delays, apod, x, y, z, nf):
    delays, dp = _d(delays)
    apod, ap = _d(apod)
    T, N = delays.shape
    x, xp = _d(x)
    y, yp = _opt(y)
    z, zp = _d(z)
    out = np.zeros((T, len(x)))
    lib().oracle_pfield(C.byref(params(cfg)), T, dp, ap, len(x), xp, yp, zp, int(nf),
                        out.ctypes.data_as(_D))
    return out


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
