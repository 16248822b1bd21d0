#!/usr/bin/env python
"""Benchmark of the SIMUS RF hot path on one GB300 (replicas on N GPUs under torchrun).

One step = one ``simus_rf`` call over the whole workload: transmit weights, Green's
terms + transmit and receive contractions, chunk reduction with the transfer factor,
inverse DFT to RF time signals.  Metric: Green's terms per second, one term being one
(frequency bin x scatterer x sub-element x transmit).

The default run times the 31-transmit convex workload on the FP16 tensor-core path (the
headline), then the plain FP32 path on the same workload, and then, briefly, the other
workloads as sub-records of the same line (``other_configs``): the 64-element focused
and 128-element plane-wave cases on the plain path, the gradient workload (forward and
adjoint), the ragged batch at 5 % of its scatterers under graph replay, and the convex
workload with BF16 operands.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--path P]
  python bench.py --impl reference ...     # the FP64 CPU oracle on a bounded sample

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2102_02738_gb300 import phantoms as ph  # noqa: E402

# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the dominant kernel, from
# the ncu capture summarised in profiles/ (per launch; absent where the kernel changed
# after the capture or none was taken)
NCU_TRAFFIC = {("diverging-convex-128", "tc_f16", 100000): 50.636544e6 + 223.560448e6,
               ("planewave-linear-128", "plain", 20003): 1.477632e6 + 0.005120e6}
# thread instructions per unique Green's term of the dominant kernel, from the same
# workloads' full captures (smsp__inst_executed.sum x 32 / unique terms); used for the
# issue-slot fraction
INST_PER_TERM = {("diverging-convex-128", "tc_f16", 100000): 3.1100394648e10 * 32 / (864 * 100000 * 256),
                 ("planewave-linear-128", "plain", 20003): 1.633e10 * 32 / (763 * 20003 * 384)}
# k_pfield on the 201 x 201 L11-5v grid (15 frequency chunks): DRAM read + write per launch
PFIELD_TRAFFIC = 1.250048e6
METRIC = "Green's terms/s (freq x scatterer x sub-elem x tx)"
WORKLOADS = {
    "planewave-linear-128": ph.planewave_linear_128,
    "diverging-convex-128": ph.diverging_convex_128,
    "focused-linear-64": ph.focused_linear_64,
    "planewave-linear-128-grad": ph.planewave_linear_128_grad,
    "ragged-batch": ph.ragged_batch,
    "planewave-linear-128-2d": ph.planewave_linear_128_2d,
    "diverging-convex-128-3d": ph.diverging_convex_128_3d,
    "pfield-l11-5v": ph.pfield_l11_5v,
}
DEFAULT_WORKLOAD = "diverging-convex-128"
DEFAULT_PATH = {"planewave-linear-128": "plain", "focused-linear-64": "plain",
                "planewave-linear-128-2d": "plain", "diverging-convex-128-3d": "tc_f16",
                "planewave-linear-128-grad": "plain", "diverging-convex-128": "tc_f16"}
# Per-term instruction budget of the Green's term (FP32 pipe, MUFU) used for the ALU
# roofline: 85 FP32-pipe instructions + 12 MUFU per (bin, scatterer, sub-element).
FP32_PER_TERM, MUFU_PER_TERM = 85, 12


def metric_terms(w, plan_info) -> float:
    return float(plan_info["n_bins"]) * w.n_scat * plan_info["n_sub"] * w.cfg["n_elements"] * w.n_tx


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_terms(n_sm: int, mhz: float) -> float:
    clk = mhz * 1e6
    return min(n_sm * 128 * clk / FP32_PER_TERM, n_sm * 16 * clk / MUFU_PER_TERM)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for ln in fh:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows
                                    if r[3].replace(".", "").isdigit()), default=None)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(v, ws):
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------- CPU oracle
def oracle_sample(w, target_s=12.0, max_bins=None, bins=None):
    """Time the oracle's RF spectrum on a subset of kept bins (all scatterers, all
    transmits); returns (terms/s, seconds, bins used, threads, bin list, spectrum)."""
    from oracle import oracle
    lo, hi, nb = oracle.bins(w.cfg)
    nu = oracle.nsub(w.cfg)
    per_bin = w.n_scat * nu * w.cfg["n_elements"] * w.n_tx
    cores = len(os.sched_getaffinity(0))
    # calibrate on as many bins as there are cores (one bin per thread)
    k = max(1, min(nb, cores if bins is None else bins))
    qs = np.linspace(lo, hi, k).round().astype(int)
    t0 = time.perf_counter()
    X = oracle.rf_spectrum(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc, qs)
    dt = time.perf_counter() - t0
    if dt < target_s and bins is None:
        k2 = int(min(nb, max(k, k * target_s / max(dt, 1e-3))))
        k2 = (k2 // cores) * cores or k2
        if max_bins:
            k2 = min(k2, max_bins)
        if k2 > k:
            qs = np.linspace(lo, hi, k2).round().astype(int)
            t0 = time.perf_counter()
            X = oracle.rf_spectrum(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc, qs)
            dt = time.perf_counter() - t0
            k = k2
    return k * per_bin / dt, dt, k, cores, qs, X


def workload_config(name, w, n_bins, n_sub):
    """The workload description both arms print (the same dict for the same workload)."""
    N = w.cfg["n_elements"]
    return {"workload": name, "scatterers": w.n_scat, "transmits": w.n_tx, "elements": N,
            "sub_elements": n_sub, "bins": n_bins, "rf_samples": w.cfg["n_samples"],
            "terms_per_step": float(n_bins) * w.n_scat * n_sub * N * w.n_tx,
            "l2": "GPU arm: flushed between timed steps (256 MB write); CPU arm: no GPU"}


def run_reference(args, rank, ws):
    if rank != 0:
        return
    w = WORKLOADS[args.workload]()
    from oracle import oracle
    lo, hi, nb = oracle.bins(w.cfg)
    nu = oracle.nsub(w.cfg)
    per_bin = w.n_scat * nu * w.cfg["n_elements"] * w.n_tx
    cores = len(os.sched_getaffinity(0))
    # each step: a fixed bin subset of at least one bin per thread (the oracle runs its
    # bins in parallel), sized for ~3 s where a bin per thread is faster than that
    _, dt1, k1, _, _, _ = oracle_sample(w, target_s=0.0)
    per_step_bins = max(k1, min(nb, int(k1 * 3.0 / max(dt1, 1e-3))))
    per_step_bins = max(k1, (per_step_bins // k1) * k1)
    qs = np.linspace(lo, hi, per_step_bins).round().astype(int)
    for _ in range(args.warmup):
        oracle.rf_spectrum(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc, qs[:max(1, len(qs) // 4)])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rf_spectrum(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc, qs)
    dt = time.perf_counter() - t0
    terms = len(qs) * per_bin * args.steps
    value = terms / dt
    sample = (f"{len(qs)} of {nb} kept bins per step, all {w.n_scat} scatterers, "
              f"{w.n_tx} transmits (RF spectrum, FP64)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "terms/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "path": "fp64-cpu-oracle",
            "config": workload_config(args.workload, w, nb, nu),
            "cpu_baseline": {"value": value, "unit": "terms/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- ours
class Ctx:
    """Device, stream, library handle and peaks shared by the measurements of one run."""

    def __init__(self, local, ws):
        import torch
        from paper_2102_02738_gb300 import build as libbuild
        libbuild.build()
        from paper_2102_02738_gb300 import simus
        torch.cuda.set_device(local)
        self.torch, self.simus, self.local, self.ws = torch, simus, local, ws
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.current_stream()
        self.peaks, self.peak_src = measured_peaks()
        self.n_sm = torch.cuda.get_device_properties(self.dev).multi_processor_count
        self.mhz = float(self.peaks.get("sm_max_mhz", 2070.0))
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=self.dev)

    def timed(self, step, steps, warmup, plans=(), flush=True):
        """W untimed warm-up steps, then K steps each bracketed by CUDA events on the
        launching stream (L2 flushed before each, untimed); the clocks are sampled during
        the timed steps.  Returns per-step ms (max over ranks of the total / K for the
        aggregate), per-step stage timings of each plan, launches and clocks."""
        torch, simus = self.torch, self.simus
        for _ in range(max(warmup, 0)):
            step()
        torch.cuda.synchronize()
        for p in plans:
            simus.simus_plan_set_profiling(p.handle, True)
        clocks = ClockSampler(self.local)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        stages = [[] for _ in plans]
        launches0 = simus.simus_kernel_launches()
        clocks.start()
        time.sleep(0.5)                             # let the sampler come up
        barrier(self.ws)
        torch.cuda.synchronize()
        for i in range(steps):
            if flush:
                self.flush.fill_(float(i))        # evict L2 between timed steps (untimed)
            ev[i][0].record(self.stream)
            step()
            ev[i][1].record(self.stream)
            for j, p in enumerate(plans):
                stages[j].append(simus.simus_plan_get_timings(p.handle))
        torch.cuda.synchronize()
        barrier(self.ws)
        launches = simus.simus_kernel_launches() - launches0
        clk = clocks.stop()
        for p in plans:
            simus.simus_plan_set_profiling(p.handle, False)
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, stages, launches, clk

    def alu_peak(self):
        return alu_peak_terms(self.n_sm, self.mhz)

    def issue_frac(self, achieved, key):
        """Fraction of the issue slots (one warp instruction per SMSP per cycle) the
        kernel's measured instruction count per unique term takes at the achieved rate."""
        ipt = INST_PER_TERM.get(key)
        if ipt is None:
            return None, None
        return achieved * ipt / 32.0 / (self.n_sm * 4 * self.mhz * 1e6), ipt


def dtype_of(path):
    return "f32" if path == "plain" else ("f32+f16" if path == "tc_f16" else "f32+bf16")


def measure_rf(ctx, name, w, path, steps, warmup, *, cpu_seconds=None, e2e=True,
               tuning=None, oracle_ref=None, oracle_bins=None):
    """One simus_rf per step over the whole workload.  Returns the JSON line and the
    device tensors, plan and oracle sample for follow-up measurements."""
    torch, simus = ctx.torch, ctx.simus
    keys = ("delays", "apod", "x", "z", "rc") + (("y",) if w.y is not None else ())
    host = {k: np.ascontiguousarray(getattr(w, k)) for k in keys}
    d = {k: torch.from_numpy(v).to(ctx.dev) for k, v in host.items()}
    plan = simus.Plan(w.cfg, path=path)
    if tuning:
        plan.set_tuning(**tuning)
    info = plan.info
    T, N, nt = w.n_tx, w.cfg["n_elements"], info["n_samples"]
    rf = torch.empty((T, N, nt), device=ctx.dev)
    terms = metric_terms(w, info)
    # Green's terms one launch generates: once per bin for all transmits (tensor-core and
    # multi-transmit plain kernels), once per transmit only for a single transmit
    unique_per_launch = terms / T

    def step():
        plan.rf(d["delays"], d["apod"], d["x"], d.get("y"), d["z"], d["rc"], out=rf,
                stream=ctx.stream)

    step_ms, stages, launches, clk = ctx.timed(step, steps, warmup, plans=[plan])
    total_ms = allreduce_max(sum(step_ms), ctx.ws)
    ms_per_step = total_ms / steps
    value = terms * ctx.ws / (ms_per_step / 1e3)
    kern_ms = statistics.mean(s["green_contract"] for s in stages[0])
    achieved = unique_per_launch / (kern_ms / 1e3)
    peak = ctx.alu_peak()
    key = (name, path, w.n_scat)
    issue, ipt = ctx.issue_frac(achieved, key)
    line = {
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": ctx.ws,
        "steps": steps, "warmup": warmup, "ms_per_step": ms_per_step,
        "ms_per_step_median": statistics.median(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_of(path), "data": "synthetic", "path": path,
        "config": workload_config(name, w, info["n_bins"], info["n_sub"]),
        "roofline": {"bound": "alu", "kernel": "green+contraction",
                     "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gterm/s",
                     "frac": achieved / peak,
                     "traffic": NCU_TRAFFIC.get(key),
                     "peak_source": f"{ctx.peak_src}: min(SMs*128*clk/{FP32_PER_TERM}, "
                                    f"SMs*16*clk/{MUFU_PER_TERM}), {ctx.n_sm} SMs at "
                                    f"{ctx.mhz} MHz",
                     "issue_frac": issue,
                     "inst_per_term": ipt,
                     "issue_source": ("thread instructions per unique term from the ncu "
                                      "capture of this kernel (smsp__inst_executed.sum x 32 / "
                                      "terms); issue slots = SMs x 4 SMSPs x clk"
                                      if ipt else "no capture of the current kernel"),
                     "kernel_ms": kern_ms},
        "stages_ms": {k: statistics.mean(s[k] for s in stages[0]) for k in simus.STAGES},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if tuning:
        line["tuning"] = dict(tuning)
    if e2e:
        # end to end through the C ABI from pinned host buffers
        pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
        rf_host = torch.empty((T, N, nt), dtype=torch.float32).pin_memory()
        h2d = sum(v.numel() * 4 for v in pinned.values())
        d2h = rf_host.numel() * 4
        e2e_steps = max(1, min(steps, 5))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_ms = 0.0
        for i in range(e2e_steps):
            ctx.flush.fill_(float(i))
            e0.record(ctx.stream)
            for k in pinned:
                d[k].copy_(pinned[k], non_blocking=True)
            step()
            rf_host.copy_(rf, non_blocking=True)
            e1.record(ctx.stream)
            e1.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        e2e_ms = allreduce_max(e2e_ms, ctx.ws) / e2e_steps
        line["e2e"] = {"value": terms * ctx.ws / (e2e_ms / 1e3), "unit": "terms/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    ref = oracle_ref
    if ref is None and cpu_seconds is not None and ctx.ws == 1:
        v, dt, k, cores, qs, Xo = oracle_sample(w, target_s=cpu_seconds, bins=oracle_bins)
        ref = (qs, Xo)
        line["cpu_baseline"] = {
            "value": v, "unit": "terms/s", "cores": cores, "kind": "oracle",
            "sample": f"RF spectrum at {k} of {info['n_bins']} kept bins, all "
                      f"{w.n_scat} scatterers and {T} transmits, FP64, {dt:.1f} s"}
    if ref is not None:
        qs, Xo = ref
        spec = plan.rf_spectrum(d["delays"], d["apod"], d["x"], d.get("y"), d["z"], d["rc"])
        Xg = spec.cpu().numpy()[..., qs - info["q_lo"]]
        line["accuracy"] = {
            "rel_l2_vs_fp64_oracle": float(np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo)),
            "compared": f"RF spectra X_q(e,t) at {len(qs)} sampled bins, every element and "
                        f"transmit", "tolerance": 1e-5 if path == "plain" else 2e-3}
    return line, {"plan": plan, "d": d, "rf": rf, "terms": terms, "ref": ref}


def measure_plain_compare(ctx, w, st, steps):
    """The plain FP32 path on the same workload and device tensors, timed like the
    headline (warm-up, L2 flush, CUDA events per step); median and spread."""
    simus = ctx.simus
    d, rf = st["d"], st["rf"]
    pplan = simus.Plan(w.cfg, path="plain")

    def step():
        pplan.rf(d["delays"], d["apod"], d["x"], d.get("y"), d["z"], d["rc"], out=rf,
                 stream=ctx.stream)

    ms, stages, _, clk = ctx.timed(step, steps, 3, plans=[pplan])
    med = statistics.median(ms)
    info = pplan.info
    pplan.close()
    kern = statistics.median(s["green_contract"] for s in stages[0])
    # the plain kernel's own budget per (bin, scatterer): M Green's terms at 85 FP32-pipe
    # instructions and the two complex contractions over (element, transmit) of Eq. 29 and
    # Eq. 32 at 4 FMA each, on the 128 FP32 lanes of an SM
    M, N, T = info["n_sub"] * info["n_elements"], info["n_elements"], w.n_tx
    pairs = float(info["n_bins"]) * w.n_scat
    peak = ctx.n_sm * ctx.mhz * 1e6 * 128.0 / (FP32_PER_TERM * M + 8.0 * N * T)
    return {"value": st["terms"] / (med / 1e3), "unit": "terms/s", "steps": steps,
            "ms_per_step_median": med, "ms_per_step_min": min(ms), "ms_per_step_max": max(ms),
            "kernel_ms_median": kern,
            "roofline": {"bound": "alu", "achieved": pairs / (kern / 1e3) / 1e9, "peak": peak / 1e9,
                         "unit": "G(bin x scatterer)/s", "frac": pairs / (kern / 1e3) / peak,
                         "peak_source": f"SMs*clk*128 / (85 M + 8 N T), M={M}, N={N}, T={T}"},
            "clocks": clk}


def measure_batch(ctx, n_sims, scale, path, steps, warmup):
    """Ragged batch: every simulation in one persistent tensor-core launch per step; the
    whole simus_batch_rf call is captured once in a CUDA graph and replayed."""
    torch, simus = ctx.torch, ctx.simus
    sims = ph.ragged_batch(n_sims=n_sims, scale=scale)
    plans = [simus.Plan(w.cfg, path=path) for w in sims]
    txs = [(torch.from_numpy(w.delays).to(ctx.dev), torch.from_numpy(w.apod).to(ctx.dev))
           for w in sims]
    scs = [(torch.from_numpy(w.x).to(ctx.dev), None, torch.from_numpy(w.z).to(ctx.dev),
            torch.from_numpy(w.rc).to(ctx.dev)) for w in sims]
    rfs = [torch.empty((w.n_tx, w.cfg["n_elements"], p.info["n_samples"]), device=ctx.dev)
           for w, p in zip(sims, plans)]
    terms = sum(float(p.info["n_bins"]) * w.n_scat * p.info["n_sub"] * w.cfg["n_elements"] * w.n_tx
                for w, p in zip(sims, plans))
    unique = sum(float(p.info["n_bins"]) * w.n_scat * p.info["n_sub"] * w.cfg["n_elements"]
                 for w, p in zip(sims, plans))
    st = torch.cuda.Stream(device=ctx.dev)
    handles = [p.handle for p in plans]
    with torch.cuda.stream(st):
        simus.simus_batch_rf(handles, txs, scs, rfs, st)            # sizes workspaces
    st.synchronize()
    l0 = simus.simus_kernel_launches()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        simus.simus_batch_rf(handles, txs, scs, rfs, st)
    per_replay = simus.simus_kernel_launches() - l0
    # inputs and outputs of the batch exceed L2 at full scale; the replay is timed as is
    ms, _, _, clk = ctx.timed(g.replay, steps, warmup, flush=scale < 0.5)
    ms_step = allreduce_max(sum(ms), ctx.ws) / steps
    peak = ctx.alu_peak()
    line = {"metric": METRIC, "value": terms * ctx.ws / (ms_step / 1e3), "unit": "terms/s",
            "n_gpus": ctx.ws, "steps": steps, "warmup": warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(path), "data": "synthetic", "path": path,
            "config": {"workload": "ragged-batch", "sims": len(sims), "scale": scale,
                       "scatterers_total": int(sum(w.n_scat for w in sims)),
                       "elements": [min(w.cfg["n_elements"] for w in sims), max(w.cfg["n_elements"] for w in sims)],
                       "transmits": [min(w.n_tx for w in sims), max(w.n_tx for w in sims)],
                       "terms_per_step": terms, "unique_terms_per_step": unique,
                       "execution": "one persistent launch per step, captured CUDA graph",
                       "l2": ("inputs and outputs exceed L2" if scale >= 0.5 else
                              "flushed between timed steps (256 MB write)")},
            "roofline": {"bound": "alu", "achieved": unique / (ms_step / 1e3) / 1e9, "peak": peak / 1e9,
                         "unit": "Gterm/s", "frac": unique / (ms_step / 1e3) / peak,
                         "note": "whole step (weights + persistent kernel + reductions + iDFTs)",
                         "peak_source": ctx.peak_src},
            "gpu_launches": per_replay * steps, "clocks": clk}
    for p in plans:
        p.close()
    return line


def measure_grad(ctx, steps, warmup, path="plain", n_scat=0, accuracy=True):
    """Forward RF plus the adjoint (simus_rf_grad) of the RF misfit L = ||RF - RF_target||^2,
    FP32.  The roofline is that of k_grad, which forms g, dg/dX and dg/dZ once per (bin,
    scatterer, sub-element) for all transmits, against the forward-term ALU budget."""
    torch, simus = ctx.torch, ctx.simus
    w = ph.planewave_linear_128_grad(**({"n_scat": n_scat} if n_scat else {}))
    plan = simus.Plan(w.cfg, path=path)
    names = ("delays", "apod", "x", "z", "rc")
    host = {k: np.ascontiguousarray(getattr(w, k), np.float32) for k in names}
    d = {k: torch.from_numpy(v).to(ctx.dev) for k, v in host.items()}
    tgt = plan.rf(d["delays"], d["apod"], torch.from_numpy(w.extra["x_target"]).to(ctx.dev), None,
                  torch.from_numpy(w.extra["z_target"]).to(ctx.dev), d["rc"])
    info = plan.info
    M = info["n_sub"] * w.cfg["n_elements"]
    terms = float(info["n_bins"]) * w.n_scat * M * w.n_tx
    fwd, bwd = [], []

    def step(record=False):
        rf = plan.rf(d["delays"], d["apod"], d["x"], None, d["z"], d["rc"])
        if record:
            fwd.append(simus.simus_plan_get_timings(plan.handle))
        drf = 2.0 * (rf - tgt)
        g = plan.rf_grad(d["delays"], d["apod"], d["x"], None, d["z"], d["rc"], drf)
        if record:
            bwd.append(simus.simus_plan_get_timings(plan.handle))
        return g

    ms, _, launches, clk = ctx.timed(lambda: step(True), steps, warmup, plans=[plan])
    fwd, bwd = fwd[-steps:], bwd[-steps:]
    ms_step = allreduce_max(sum(ms), ctx.ws) / steps
    fwd_ms = statistics.mean(sum(t.values()) for t in fwd)
    bwd_ms = statistics.mean(sum(t.values()) for t in bwd)
    grad_ms = statistics.mean(t["gradient"] for t in bwd)
    # k_grad's budget per (bin, scatterer): M Green's terms at the forward-term count (85
    # FP32-pipe instructions + 12 SFU; their X/Z derivatives are not counted) and six complex
    # contractions over (element, transmit) of 4 FMA each (P, dP/dX, dP/dZ and the three
    # receive-side sums against the adjoint spectrum)
    n_el = w.cfg["n_elements"]
    cyc_pair = max((FP32_PER_TERM * M + 24.0 * n_el * w.n_tx) / 128.0, MUFU_PER_TERM * M / 16.0)
    peak_pairs = ctx.n_sm * ctx.mhz * 1e6 / cyc_pair
    pairs = float(info["n_bins"]) * w.n_scat
    achieved = pairs / (grad_ms / 1e3)
    # end to end: scatterers and transmit settings in from pinned host memory, the four
    # gradients out to pinned host memory
    pin = {k: torch.from_numpy(host[k]).pin_memory() for k in names}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    outs_h = None
    e2e_ms = 0.0
    n_e2e = max(1, min(steps, 5))
    for i in range(n_e2e):
        ctx.flush.fill_(float(i))
        e0.record(ctx.stream)
        for k in names:
            d[k].copy_(pin[k], non_blocking=True)
        g = step()
        if outs_h is None:
            outs_h = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in g.items()}
        for k, v in g.items():
            outs_h[k].copy_(v, non_blocking=True)
        e1.record(ctx.stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = allreduce_max(e2e_ms, ctx.ws) / n_e2e
    line = {"metric": METRIC + ", forward + adjoint", "value": terms * ctx.ws / (ms_step / 1e3),
            "unit": "terms/s", "n_gpus": ctx.ws, "steps": steps, "warmup": warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "path": path,
            "config": {"workload": "planewave-linear-128-grad", "forward_path": path,
                       "scatterers": w.n_scat, "transmits": w.n_tx, "bins": info["n_bins"],
                       "sub_elements_total": M, "terms_per_step": terms,
                       "l2": "flushed between timed steps (256 MB write)"},
            "roofline": {"bound": "alu", "kernel": "k_grad", "achieved": achieved / 1e9,
                         "peak": peak_pairs / 1e9, "unit": "G(bin x scatterer)/s",
                         "frac": achieved / peak_pairs, "traffic": None, "kernel_ms": grad_ms,
                         "peak_source": f"SMs*clk / max((85 M + 24 N T) / 128, 12 M / 16) cycles per "
                                        f"(bin, scatterer), M={M}, N={n_el}, T={w.n_tx}, "
                                        f"{ctx.n_sm} SMs at {ctx.mhz} MHz"},
            "forward_ms": fwd_ms, "adjoint_ms": bwd_ms,
            "adjoint_stages_ms": {k: statistics.mean(t[k] for t in bwd) for k in simus.STAGES},
            "e2e": {"value": terms * ctx.ws / (e2e_ms / 1e3), "unit": "terms/s",
                    "h2d_bytes_per_step": sum(v.numel() * 4 for v in pin.values()),
                    "d2h_bytes_per_step": sum(v.numel() * 4 for v in outs_h.values())},
            "gpu_launches": launches, "clocks": clk}
    if accuracy and ctx.ws == 1:
        # the FP64 oracle's adjoint for a sample of scatterers from a seeded upstream
        # gradient: per-scatterer gradients depend only on it and the scatterer
        from oracle import oracle as orc
        T, nt = w.n_tx, info["n_samples"]
        drf = ph.normal(1004, 31, T * n_el * nt).reshape(T, n_el, nt).astype(np.float32)
        g = plan.rf_grad(d["delays"], d["apod"], d["x"], None, d["z"], d["rc"],
                         torch.from_numpy(drf).to(ctx.dev))
        torch.cuda.synchronize()
        sel = np.linspace(0, w.n_scat - 1, 24).astype(np.int64)
        t0 = time.time()
        gR, gx, gz, _ = orc.rf_grad(w.cfg, host["delays"], host["apod"], host["x"][sel], None,
                                    host["z"][sel], host["rc"][sel], drf)
        dt = time.time() - t0
        line["cpu_baseline"] = {"value": float(info["n_bins"]) * sel.size * M * w.n_tx / dt,
                                "unit": "terms/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                                "sample": f"adjoint only, {sel.size} of {w.n_scat} scatterers, all bins and "
                                          f"transmits, FP64, including its DFT of the upstream gradient, "
                                          f"{dt:.1f} s"}
        acc = {}
        for k, ref in (("rc", gR), ("x", gx), ("z", gz)):
            got = g[k].double().cpu().numpy()[sel]
            acc[k] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        line["accuracy"] = {"rel_l2_vs_fp64_oracle": acc, "tolerance": 1e-5,
                            "compared": f"dL/dR, dL/dX, dL/dZ at {sel.size} sampled scatterers of "
                                        f"the full workload, seeded upstream gradient"}
    plan.close()
    return line


def measure_pfield(ctx, steps, warmup, accuracy=True, n_check=60):
    """RMS field (Eq. 41-42) of the Fig. 10 L11-5v setup on a 201 x 201 x-z grid, FP32."""
    torch, simus = ctx.torch, ctx.simus
    w = ph.pfield_l11_5v()
    cfg = w.cfg
    plan = simus.Plan(cfg, path="plain")
    xe, ze = ph.element_centres(cfg)
    r_max = float(np.max(np.hypot(w.x[:, None] - xe[None, :], w.z[:, None] - ze[None, :]))) + cfg["width"]
    nf = simus.simus_pfield_nfreq(cfg, r_max, float(w.delays.max()))
    host = {k: np.ascontiguousarray(getattr(w, k)) for k in ("delays", "apod", "x", "z")}
    d = {k: torch.from_numpy(v).to(ctx.dev) for k, v in host.items()}
    npts = w.x.size
    out = torch.empty((w.n_tx, npts), device=ctx.dev)
    M = plan.info["n_sub"] * cfg["n_elements"]
    terms = float(npts) * nf * M * w.n_tx

    def step():
        plan.pfield(d["delays"], d["apod"], d["x"], None, d["z"], nf, out=out, stream=ctx.stream)

    ms, stages, launches, clk = ctx.timed(step, steps, warmup, plans=[plan])
    ms_per_step = allreduce_max(sum(ms), ctx.ws) / steps
    kern_ms = statistics.mean(s["pfield"] for s in stages[0])
    peak = ctx.alu_peak()
    achieved = terms / (kern_ms / 1e3)
    # end to end: grid coordinates in, field out, through pinned host buffers
    pin = {k: torch.from_numpy(host[k]).pin_memory() for k in ("x", "z")}
    out_h = torch.empty((w.n_tx, npts), dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    n_e2e = max(1, min(steps, 5))
    for i in range(n_e2e):
        ctx.flush.fill_(float(i))
        e0.record(ctx.stream)
        for k in pin:
            d[k].copy_(pin[k], non_blocking=True)
        step()
        out_h.copy_(out, non_blocking=True)
        e1.record(ctx.stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = allreduce_max(e2e_ms, ctx.ws) / n_e2e
    line = {"metric": METRIC.replace("scatterer", "field point"), "value": terms * ctx.ws / (ms_per_step / 1e3),
            "unit": "terms/s", "n_gpus": ctx.ws, "steps": steps, "warmup": warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "path": "plain",
            "config": {"workload": "pfield-l11-5v", "points": npts, "frequencies": nf,
                       "sub_elements_total": M, "transmits": w.n_tx, "terms_per_step": terms,
                       "l2": "flushed between timed steps (256 MB write)"},
            "roofline": {"bound": "alu", "kernel": "k_pfield", "achieved": achieved / 1e9,
                         "peak": peak / 1e9, "unit": "Gterm/s", "frac": achieved / peak,
                         "traffic": PFIELD_TRAFFIC, "kernel_ms": kern_ms},
            "e2e": {"value": terms * ctx.ws / (e2e_ms / 1e3), "unit": "terms/s",
                    "h2d_bytes_per_step": sum(v.numel() * 4 for v in pin.values()),
                    "d2h_bytes_per_step": out_h.numel() * 4},
            "gpu_launches": launches, "clocks": clk}
    if accuracy and ctx.ws == 1:
        from oracle import oracle as orc
        sel = np.linspace(0, npts - 1, n_check).astype(np.int64)
        t0 = time.time()
        ref = orc.pfield(cfg, w.delays, w.apod, w.x[sel], None, w.z[sel], nf)
        dt = time.time() - t0
        got = out.cpu().numpy()[:, sel]
        line["cpu_baseline"] = {"value": float(sel.size) * nf * M * w.n_tx / dt, "unit": "terms/s",
                                "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                                "sample": f"{sel.size} of {npts} grid points, all {nf} frequencies, FP64, {dt:.1f} s"}
        line["accuracy"] = {"rel_l2_vs_fp64_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                            "compared": f"RMS pressure at the {sel.size} sampled points", "tolerance": 1e-5}
    plan.close()
    return line


SUB_KEYS = ("ms_per_step", "ms_per_step_median", "value", "unit", "steps", "path", "dtype",
            "forward_ms", "adjoint_ms", "accuracy", "tuning")


def compact(line):
    """The sub-record of another workload inside the headline line."""
    out = {k: line[k] for k in SUB_KEYS if k in line}
    out["config"] = {k: v for k, v in line["config"].items() if k != "l2"}
    r = line["roofline"]
    out["roofline"] = {k: r[k] for k in ("kernel", "achieved", "peak", "unit", "frac", "kernel_ms",
                                         "issue_frac") if k in r}
    out["clocks"] = {k: line["clocks"].get(k) for k in ("sm_mhz", "reasons")}
    return out


def other_configs(ctx, headline_ref):
    """The other workloads, measured briefly after the headline (single GPU only)."""
    out = {}
    t0 = time.time()
    w = ph.focused_linear_64()
    line, st = measure_rf(ctx, "focused-linear-64", w, "plain", 10, 3, cpu_seconds=1.0, e2e=False)
    st["plan"].close()
    out["focused-linear-64"] = compact(line)
    w = ph.planewave_linear_128()
    line, st = measure_rf(ctx, "planewave-linear-128", w, "plain", 5, 2, cpu_seconds=2.0, e2e=False)
    st["plan"].close()
    out["planewave-linear-128"] = compact(line)
    out["planewave-linear-128-grad"] = compact(measure_grad(ctx, 5, 2))
    out["ragged-batch-x0.05"] = compact(measure_batch(ctx, 256, 0.05, "tc_f16", 2, 3))
    # the paper's other models on the same kernels: RMS field (Eq. 41-42), the 2-D model
    # (Section V) and scatterers off the azimuth plane (Eq. 14 with Y != 0)
    out["pfield-l11-5v"] = compact(measure_pfield(ctx, 5, 2, n_check=20))
    w = ph.planewave_linear_128_2d()
    line, st = measure_rf(ctx, "planewave-linear-128-2d", w, "plain", 5, 2, cpu_seconds=0.0, e2e=False)
    st["plan"].close()
    out["planewave-linear-128-2d"] = compact(line)
    w = ph.diverging_convex_128_3d()
    # (no oracle sample here: with Y != 0 one bin takes the oracle ~14 s; the parity tests
    # cover this path)
    line, st = measure_rf(ctx, "diverging-convex-128-3d", w, "tc_f16", 3, 3, e2e=False)
    st["plan"].close()
    out["diverging-convex-128-3d"] = compact(line)
    w = WORKLOADS[DEFAULT_WORKLOAD]()
    line, st = measure_rf(ctx, DEFAULT_WORKLOAD, w, "tc_bf16", 5, 2, e2e=False,
                          oracle_ref=headline_ref)
    st["plan"].close()
    out[DEFAULT_WORKLOAD + "-bf16"] = compact(line)
    out["seconds"] = time.time() - t0
    return out


def run_ours(args, rank, ws, local):
    ctx = Ctx(local, ws)
    tuning = dict(kv.split("=") for kv in args.tune) if args.tune else None
    tuning = {k: int(v) for k, v in tuning.items()} if tuning else None
    if args.workload == "ragged-batch":
        line = measure_batch(ctx, args.n_sims, args.scale, args.path or "tc_f16", args.steps,
                             args.warmup)
    elif args.workload == "planewave-linear-128-grad":
        line = measure_grad(ctx, args.steps, args.warmup, args.path or "plain", args.n_scat,
                            accuracy=not args.no_cpu_baseline)
    elif args.workload == "pfield-l11-5v":
        line = measure_pfield(ctx, args.steps, args.warmup, accuracy=not args.no_cpu_baseline)
    else:
        w = WORKLOADS[args.workload](**({"n_scat": args.n_scat} if args.n_scat else {}))
        path = args.path or DEFAULT_PATH[args.workload]
        line, st = measure_rf(ctx, args.workload, w, path, args.steps, args.warmup,
                              cpu_seconds=None if args.no_cpu_baseline else args.cpu_seconds,
                              tuning=tuning)
        if path != "plain" and not args.no_plain_compare:
            pc = measure_plain_compare(ctx, w, st, max(5, min(args.steps, 10)))
            pc["speedup_of_this_path"] = pc["ms_per_step_median"] / line["ms_per_step_median"]
            line["plain_f32_same_workload"] = pc
        st["plan"].close()
        if (args.workload == DEFAULT_WORKLOAD and not args.n_scat and ws == 1 and not tuning
                and not args.no_other_configs):
            line["other_configs"] = other_configs(ctx, st["ref"])
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--path", default=None, choices=[None, "plain", "tc_f16", "tc_bf16"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain-compare", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="headline workload only (no sub-records of the other workloads)")
    ap.add_argument("--tune", nargs="*", default=None,
                    help="tensor-core tuning overrides, e.g. delta_table=0 pair=1")
    ap.add_argument("--n-scat", type=int, default=0,
                    help="override the workload's scatterer count (profiling of small cases)")
    ap.add_argument("--n-sims", type=int, default=256, help="ragged-batch: simulations")
    ap.add_argument("--scale", type=float, default=1.0, help="ragged-batch: scatterer count scale")
    args = ap.parse_args()
    rank, ws, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_ours(args, rank, ws, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
