"""Thin Python binding of the C ABI in ``include/simus.h`` (ctypes; argument marshalling
only -- every step of the computation runs in the CUDA library).

Tensors are torch CUDA tensors (float32, contiguous); PyTorch provides device memory
and streams.  Functions carry the C names (``simus_rf``, ``simus_pfield``, ...);
:class:`Plan` wraps a plan handle, and :class:`RFFunction` is the autograd wrapper of
``simus_rf`` / ``simus_rf_grad``.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2102_02738_gb300.build``); importing this module raises if it is
missing.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import torch

from . import build as _build

PATH_PLAIN_F32, PATH_TC_F16, PATH_TC_BF16 = 0, 1, 2
_PATHS = {"plain": 0, "f32": 0, "tc_f16": 1, "f16": 1, "tc_bf16": 2, "bf16": 2}
ERR = {0: "OK", -1: "SIMUS_ERR_ARG", -2: "SIMUS_ERR_CUDA", -3: "SIMUS_ERR_OOM",
       -4: "SIMUS_ERR_TIMEOUT", -5: "SIMUS_ERR_UNSUPPORTED"}


class SimusError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR.get(code, code)}: {msg}")
        self.code = code


class Probe(C.Structure):
    _fields_ = [("n_elements", C.c_int32), ("n_sub", C.c_int32), ("baffle", C.c_int32),
                ("two_d", C.c_int32), ("pitch", C.c_double), ("width", C.c_double),
                ("height", C.c_double), ("elev_focus", C.c_double), ("radius", C.c_double),
                ("fc", C.c_double), ("frac_bw", C.c_double), ("zeta", C.c_double)]


class Medium(C.Structure):
    _fields_ = [("c", C.c_double), ("alpha_db", C.c_double), ("fs", C.c_double),
                ("pulse", C.c_int32), ("reserved", C.c_int32), ("pulse_cycles", C.c_double)]


class Tx(C.Structure):
    _fields_ = [("n_tx", C.c_int32), ("reserved", C.c_int32), ("delays", C.c_void_p),
                ("apod", C.c_void_p)]


class Scat(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("rc", C.c_void_p)]


class PlanInfo(C.Structure):
    _fields_ = [("n_elements", C.c_int32), ("n_sub", C.c_int32), ("n_samples", C.c_int32),
                ("path", C.c_int32), ("q_lo", C.c_int32), ("q_hi", C.c_int32),
                ("n_bins", C.c_int32), ("reserved", C.c_int32), ("df", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("items_per_sm", C.c_int32), ("max_bins", C.c_int32), ("pair", C.c_int32),
                ("delta_table", C.c_int32), ("chunks", C.c_int32), ("tile_buffers", C.c_int32),
                ("depth_order", C.c_int32), ("tensor_idft", C.c_int32)]


TUNING_FIELDS = ("items_per_sm", "max_bins", "pair", "delta_table", "chunks", "tile_buffers",
                 "depth_order", "tensor_idft")


def _load():
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library not built: {_build.LIB} is missing "
                          "(run __graft_entry__.build())")
    L = C.CDLL(_build.LIB)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    L.simus_plan_create.argtypes = [C.POINTER(Probe), C.POINTER(Medium), i32, i32,
                                    C.POINTER(vp)]
    L.simus_plan_destroy.argtypes = [vp]
    L.simus_plan_destroy.restype = None
    L.simus_plan_get_info.argtypes = [vp, C.POINTER(PlanInfo)]
    L.simus_default_nt.argtypes = [C.POINTER(Probe), C.POINTER(Medium), d, d]
    L.simus_default_nt.restype = i32
    L.simus_pfield_nfreq.argtypes = [C.POINTER(Probe), C.POINTER(Medium), d, d]
    L.simus_pfield_nfreq.restype = i32
    L.simus_rf.argtypes = [vp, C.POINTER(Tx), C.POINTER(Scat), vp, vp]
    L.simus_rf_spectrum.argtypes = [vp, C.POINTER(Tx), C.POINTER(Scat), vp, vp]
    L.simus_pfield.argtypes = [vp, C.POINTER(Tx), i64, vp, vp, vp, i32, vp, vp]
    L.simus_rf_grad.argtypes = [vp, C.POINTER(Tx), C.POINTER(Scat), vp, vp, vp, vp, vp, vp]
    L.simus_batch_rf.argtypes = [i32, C.POINTER(vp), C.POINTER(Tx), C.POINTER(Scat),
                                 C.POINTER(vp), vp]
    L.simus_batch_rf_spectrum.argtypes = [i32, C.POINTER(vp), C.POINTER(Tx),
                                          C.POINTER(Scat), C.POINTER(vp), vp]
    L.simus_last_error.restype = C.c_char_p
    L.simus_plan_set_profiling.argtypes = [vp, i32]
    L.simus_plan_get_timings.argtypes = [vp, C.POINTER(C.c_float)]
    L.simus_plan_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.simus_plan_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.simus_kernel_launches.restype = i64
    L.simus_kernel_launches.argtypes = []
    L.simus_plan_check.argtypes = [vp]
    L.simus_plan_selftest_timeout.argtypes = [vp, i32, vp]
    L.simus_rf_noalloc.argtypes = [C.POINTER(Probe), C.POINTER(Medium), i32, C.POINTER(Tx),
                                   C.POINTER(Scat), vp, vp]
    return L


N_STAGES = 8
STAGES = ("tx_weights", "green_contract", "reduce", "idft", "pfield", "adjoint_dft",
          "gradient", "other")


lib = _load()


def _check(rc):
    if rc != 0:
        raise SimusError(rc, lib.simus_last_error().decode())
    return rc


# ------------------------------------------------------------------- marshalling
def probe_struct(cfg: dict) -> Probe:
    ef = cfg.get("elev_focus", math.inf)
    return Probe(int(cfg["n_elements"]), int(cfg.get("n_sub", 0)), int(cfg.get("baffle", 0)),
                 int(cfg.get("two_d", 0)),
                 float(cfg["pitch"]), float(cfg["width"]), float(cfg["height"]),
                 float(ef if ef is not None else math.inf), float(cfg.get("radius", 0.0)),
                 float(cfg["fc"]), float(cfg["frac_bw"]), float(cfg.get("zeta", 1.75)))


def medium_struct(cfg: dict) -> Medium:
    return Medium(float(cfg["c"]), float(cfg["alpha_db"]), float(cfg["fs"]),
                  int(cfg.get("pulse", 0)), 0, float(cfg.get("pulse_cycles", 1.0)))


def _dev(t, name, shape=None):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def tx_struct(delays, apod) -> Tx:
    T, N = delays.shape
    return Tx(T, 0, _dev(delays, "delays"), _dev(apod, "apod", (T, N)))


def scat_struct(x, y, z, rc) -> Scat:
    S = x.shape[0]
    return Scat(S, _dev(x, "x"), _dev(y, "y", (S,)), _dev(z, "z", (S,)), _dev(rc, "rc", (S,)))


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------- C-named functions
def simus_default_nt(cfg, r_max, tau_max) -> int:
    return _check_nonneg(lib.simus_default_nt(C.byref(probe_struct(cfg)),
                                              C.byref(medium_struct(cfg)), r_max, tau_max))


def simus_pfield_nfreq(cfg, r_max, tau_max) -> int:
    return _check_nonneg(lib.simus_pfield_nfreq(C.byref(probe_struct(cfg)),
                                                C.byref(medium_struct(cfg)), r_max, tau_max))


def _check_nonneg(v):
    if v < 0:
        _check(v)
    return v


def simus_plan_create(cfg: dict, n_samples: int, path=PATH_PLAIN_F32):
    h = C.c_void_p()
    _check(lib.simus_plan_create(C.byref(probe_struct(cfg)), C.byref(medium_struct(cfg)),
                                 int(n_samples), int(_PATHS.get(path, path)), C.byref(h)))
    return h


def simus_plan_destroy(h):
    lib.simus_plan_destroy(h)


def simus_plan_get_info(h) -> dict:
    info = PlanInfo()
    _check(lib.simus_plan_get_info(h, C.byref(info)))
    return {k: getattr(info, k) for k, _ in PlanInfo._fields_ if k != "reserved"}


def simus_rf(h, delays, apod, x, y, z, rc, rf, stream=None):
    _check(lib.simus_rf(h, C.byref(tx_struct(delays, apod)), C.byref(scat_struct(x, y, z, rc)),
                        _dev(rf, "rf"), _stream(stream)))


def simus_rf_spectrum(h, delays, apod, x, y, z, rc, spec, stream=None):
    _check(lib.simus_rf_spectrum(h, C.byref(tx_struct(delays, apod)),
                                 C.byref(scat_struct(x, y, z, rc)), _dev(spec, "spec"),
                                 _stream(stream)))


def simus_pfield(h, delays, apod, x, y, z, n_freq, prms, stream=None):
    _check(lib.simus_pfield(h, C.byref(tx_struct(delays, apod)), x.shape[0], _dev(x, "x"),
                            _dev(y, "y"), _dev(z, "z"), int(n_freq), _dev(prms, "prms"),
                            _stream(stream)))


def simus_rf_grad(h, delays, apod, x, y, z, rc, drf, g_rc=None, g_x=None, g_z=None,
                  g_delays=None, stream=None):
    _check(lib.simus_rf_grad(h, C.byref(tx_struct(delays, apod)),
                             C.byref(scat_struct(x, y, z, rc)), _dev(drf, "drf"),
                             _dev(g_rc, "g_rc"), _dev(g_x, "g_x"), _dev(g_z, "g_z"),
                             _dev(g_delays, "g_delays"), _stream(stream)))


def simus_plan_check(h):
    _check(lib.simus_plan_check(h))


def simus_rf_noalloc(cfg, n_samples, delays, apod, x, y, z, rc, rf, stream=None):
    """simus_rf without device allocation (fixed per-device scratch; see simus.h)."""
    _check(lib.simus_rf_noalloc(C.byref(probe_struct(cfg)), C.byref(medium_struct(cfg)),
                                int(n_samples), C.byref(tx_struct(delays, apod)),
                                C.byref(scat_struct(x, y, z, rc)), _dev(rf, "rf"),
                                _stream(stream)))


def simus_plan_set_profiling(h, enable=True):
    _check(lib.simus_plan_set_profiling(h, int(bool(enable))))


def simus_plan_get_timings(h) -> dict:
    ms = (C.c_float * N_STAGES)()
    _check(lib.simus_plan_get_timings(h, ms))
    return {name: float(v) for name, v in zip(STAGES, ms)}


def simus_plan_set_tuning(h, **values):
    """Set tensor-core launch shapes; fields not given keep their current value."""
    t = Tuning()
    _check(lib.simus_plan_get_tuning(h, t))
    for k, v in values.items():
        if k not in TUNING_FIELDS:
            raise KeyError(k)
        setattr(t, k, int(v))
    _check(lib.simus_plan_set_tuning(h, t))


def simus_plan_get_tuning(h) -> dict:
    t = Tuning()
    _check(lib.simus_plan_get_tuning(h, t))
    return {k: int(getattr(t, k)) for k in TUNING_FIELDS}


def simus_kernel_launches() -> int:
    return int(lib.simus_kernel_launches())


def simus_batch_rf(handles, txs, scats, rfs, stream=None):
    n = len(handles)
    hs = (C.c_void_p * n)(*[h.value for h in handles])
    tx = (Tx * n)(*[tx_struct(d, a) for d, a in txs])
    sc = (Scat * n)(*[scat_struct(*s) for s in scats])
    out = (C.c_void_p * n)(*[_dev(r, "rf") for r in rfs])
    _check(lib.simus_batch_rf(n, hs, tx, sc, out, _stream(stream)))


def simus_batch_rf_spectrum(handles, txs, scats, specs, stream=None):
    """specs[i]: float32 [T_i][N_i][n_bins_i][2] CUDA tensors (interleaved re, im)."""
    n = len(handles)
    hs = (C.c_void_p * n)(*[h.value for h in handles])
    tx = (Tx * n)(*[tx_struct(d, a) for d, a in txs])
    sc = (Scat * n)(*[scat_struct(*s) for s in scats])
    out = (C.c_void_p * n)(*[_dev(r, "spec") for r in specs])
    _check(lib.simus_batch_rf_spectrum(n, hs, tx, sc, out, _stream(stream)))


# ------------------------------------------------------------------------- Plan
class Plan:
    """A plan for one probe / medium / RF length / contraction path."""

    def __init__(self, cfg: dict, n_samples: int | None = None, path="plain"):
        self.cfg = dict(cfg)
        nt = int(n_samples or cfg["n_samples"])
        self.handle = simus_plan_create(cfg, nt, path)
        self.info = simus_plan_get_info(self.handle)

    def close(self):
        if self.handle is not None and self.handle.value:
            simus_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, **values):
        simus_plan_set_tuning(self.handle, **values)

    def get_tuning(self) -> dict:
        return simus_plan_get_tuning(self.handle)

    @property
    def n_bins(self):
        return self.info["n_bins"]

    @property
    def bins(self):
        return torch.arange(self.info["q_lo"], self.info["q_hi"] + 1)

    def rf(self, delays, apod, x, y, z, rc, out=None, stream=None):
        T, N = delays.shape
        if out is None:
            out = torch.empty((T, N, self.info["n_samples"]), device=x.device, dtype=torch.float32)
        simus_rf(self.handle, delays, apod, x, y, z, rc, out, stream)
        return out

    def rf_spectrum(self, delays, apod, x, y, z, rc, out=None, stream=None):
        T, N = delays.shape
        if out is None:
            out = torch.empty((T, N, self.n_bins, 2), device=x.device, dtype=torch.float32)
        simus_rf_spectrum(self.handle, delays, apod, x, y, z, rc, out, stream)
        return torch.view_as_complex(out)

    def pfield(self, delays, apod, x, y, z, n_freq, out=None, stream=None):
        T = delays.shape[0]
        if out is None:
            out = torch.empty((T, x.shape[0]), device=x.device, dtype=torch.float32)
        simus_pfield(self.handle, delays, apod, x, y, z, n_freq, out, stream)
        return out

    def rf_grad(self, delays, apod, x, y, z, rc, drf, want=("rc", "x", "z", "delays"),
                stream=None):
        S = x.shape[0]
        dev = x.device
        g = {k: (torch.empty(S, device=dev) if k in want else None) for k in ("rc", "x", "z")}
        g["delays"] = torch.empty_like(delays) if "delays" in want else None
        simus_rf_grad(self.handle, delays, apod, x, y, z, rc, drf, g["rc"], g["x"], g["z"],
                      g["delays"], stream)
        return g


class RFFunction(torch.autograd.Function):
    """rf = simus_rf(x, z, rc, delays); backward via simus_rf_grad (Green's terms are
    recomputed in the backward pass, nothing is stored but the inputs)."""

    @staticmethod
    def forward(ctx, plan: Plan, x, z, rc, delays, apod):
        ctx.plan = plan
        ctx.save_for_backward(x, z, rc, delays, apod)
        return plan.rf(delays.contiguous(), apod.contiguous(), x.contiguous(), None,
                       z.contiguous(), rc.contiguous())

    @staticmethod
    def backward(ctx, grad_rf):
        x, z, rc, delays, apod = ctx.saved_tensors
        want = []
        for name, need in zip(("x", "z", "rc", "delays"), ctx.needs_input_grad[1:5]):
            if need:
                want.append(name)
        g = ctx.plan.rf_grad(delays.contiguous(), apod.contiguous(), x.contiguous(), None,
                             z.contiguous(), rc.contiguous(), grad_rf.contiguous(), want=want)
        return None, g["x"], g["z"], g["rc"], g["delays"], None


def rf_autograd(plan: Plan, x, z, rc, delays, apod):
    return RFFunction.apply(plan, x, z, rc, delays, apod)
