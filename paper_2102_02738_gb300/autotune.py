"""Empirical autotuner for the tensor-core path's launch shapes.

For a problem shape -- device, contraction path, elements N, sub-elements nu, transmits T,
kept bins, scatterer count S rounded to a power of two -- it times candidate tunings
(`simus_tuning`: bins per work item, bins per generation pass, one or two tile buffers,
delta table, scatterer chunks; items per SM for batches) through the library's own entry points with CUDA
events, keeps the fastest and caches it in a JSON file, so later plans of the same
shape start from it without timing.  Results do not depend on the tuning beyond FP32
summation order (and the delta table's 2.3e-6 relative error), so tuning never changes
what is computed.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import torch

from . import simus

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "simus_gb300", "tuning.json")


def _bucket(n: int) -> int:
    return 1 << max(0, math.ceil(math.log2(max(1, n))))


def shape_key(plan: simus.Plan, T: int, S: int, batch: int = 1) -> str:
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    i = plan.info
    return (f"{dev}|path{i['path']}|N{i['n_elements']}|nu{i['n_sub']}|T{T}|nq{i['n_bins']}"
            f"|S{_bucket(S)}|B{batch}")


def candidates(single: bool = True):
    """Tunings to time: bins per item x bins per generation pass x tile buffers (passes of
    two or three bins) x delta table (x items per SM for batches).  Chunk counts are left
    to the library's makespan model."""
    out = []
    for mb, pair, tab in itertools.product((2, 3, 4, 6), (2, 1, 0), (1, 0)):
        for tbuf in ((2, 1) if pair > 0 else (1,)):
            base = dict(max_bins=mb, pair=pair, delta_table=tab, tile_buffers=tbuf)
            if single:
                out.append(dict(base, chunks=0))
            else:
                for ips in (2, 4, 8):
                    out.append(dict(base, items_per_sm=ips))
    return out


def _time(fn, reps: int) -> float:
    fn()                                   # warm-up (also grows the workspace)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_rf(plan: simus.Plan, delays, apod, x, y, z, rc, reps: int = 2,
            cache_path: str | None = DEFAULT_CACHE, cands=None, verbose: bool = False) -> dict:
    """Time simus_rf under each candidate tuning on these device inputs, set the fastest
    on the plan and record it in the cache.  Returns {"best": tuning, "ms": t, "all": [...]}."""
    T, S = delays.shape[0], x.shape[0]
    out = torch.empty((T, plan.info["n_elements"], plan.info["n_samples"]),
                      device=x.device, dtype=torch.float32)
    results = []
    for c in cands or candidates(single=True):
        plan.set_tuning(**c)
        ms = _time(lambda: plan.rf(delays, apod, x, y, z, rc, out=out), reps)
        results.append((ms, c))
        if verbose:
            print(f"  {c} -> {ms:.3f} ms", flush=True)
    results.sort(key=lambda r: r[0])
    best_ms, best = results[0]
    plan.set_tuning(**best)
    if cache_path:
        cache = load_cache(cache_path)
        cache[shape_key(plan, T, S)] = dict(best, ms=best_ms)
        save_cache(cache, cache_path)
    return {"best": best, "ms": best_ms, "all": [dict(c, ms=m) for m, c in results]}


def tune_batch(plans, txs, scats, rfs, reps: int = 2, cache_path: str | None = DEFAULT_CACHE,
               cands=None, verbose: bool = False) -> dict:
    """The same for one simus_batch_rf call (every plan gets the candidate; items per SM
    is read from the first plan)."""
    handles = [p.handle for p in plans]
    results = []
    for c in cands or candidates(single=False):
        for p in plans:
            p.set_tuning(**c)
        ms = _time(lambda: simus.simus_batch_rf(handles, txs, scats, rfs), reps)
        results.append((ms, c))
        if verbose:
            print(f"  {c} -> {ms:.3f} ms", flush=True)
    results.sort(key=lambda r: r[0])
    best_ms, best = results[0]
    for p in plans:
        p.set_tuning(**best)
    if cache_path:
        cache = load_cache(cache_path)
        S = sum(int(s[0].shape[0]) for s in scats)
        T = sum(int(t[0].shape[0]) for t in txs)
        cache[shape_key(plans[0], T, S, batch=len(plans))] = dict(best, ms=best_ms)
        save_cache(cache, cache_path)
    return {"best": best, "ms": best_ms, "all": [dict(c, ms=m) for m, c in results]}


def apply_cached(plan: simus.Plan, T: int, S: int, batch: int = 1,
                 cache_path: str = DEFAULT_CACHE) -> bool:
    """Set the cached tuning for this shape on the plan, if there is one."""
    entry = load_cache(cache_path).get(shape_key(plan, T, S, batch))
    if not entry:
        return False
    plan.set_tuning(**{k: v for k, v in entry.items() if k in simus.TUNING_FIELDS})
    return True
