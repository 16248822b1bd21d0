"""Checkpointed ragged batches: many independent simulations run through simus_batch_rf
in groups, each simulation's RF saved under its index, so that a rerun after an
interruption skips the simulations already finished.

The paper has no counterpart (its simulator runs one simulation per call); this is the
resume logic for long batches of the kind the ragged-batch workload describes.  Runs are
deterministic for given inputs, so a resumed batch gives the same files as an
uninterrupted one.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

INDEX = "index.json"


def _key(sims) -> str:
    """Fingerprint of the batch (configs, shapes and input bytes) stored with the index,
    so that a directory is never resumed with a different batch."""
    h = hashlib.sha256()
    for w in sims:
        h.update(json.dumps(w.cfg, sort_keys=True).encode())
        for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc):
            if a is not None:
                h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _load_index(out_dir: str, key: str) -> set:
    try:
        with open(os.path.join(out_dir, INDEX)) as f:
            idx = json.load(f)
    except (OSError, ValueError):
        return set()
    if idx.get("key") != key:
        raise ValueError(f"{out_dir} holds the results of a different batch")
    return {int(i) for i in idx.get("done", [])}


def _save_index(out_dir: str, key: str, done: set) -> None:
    tmp = os.path.join(out_dir, INDEX + ".tmp")
    with open(tmp, "w") as f:
        json.dump({"key": key, "done": sorted(done)}, f)
    os.replace(tmp, os.path.join(out_dir, INDEX))


def rf_path(out_dir: str, i: int) -> str:
    return os.path.join(out_dir, f"rf_{i:05d}.npy")


def _gpu_runner(path):
    """Default runner: one simus_batch_rf call per group, RF copied back to the host."""
    import torch
    from . import simus

    def dev(a):
        return None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()

    def run(group):
        plans = [simus.Plan(w.cfg, path=path) for w in group]
        txs = [(dev(w.delays), dev(w.apod)) for w in group]
        scs = [(dev(w.x), dev(w.y), dev(w.z), dev(w.rc)) for w in group]
        rfs = [torch.empty((w.n_tx, w.cfg["n_elements"], p.info["n_samples"]), device="cuda")
               for w, p in zip(group, plans)]
        simus.simus_batch_rf([p.handle for p in plans], txs, scs, rfs)
        rc = simus.lib.simus_plan_check(plans[0].handle)
        if rc != 0:
            raise simus.SimusError(rc, simus.lib.simus_last_error().decode())
        out = [r.cpu().numpy() for r in rfs]
        for p in plans:
            p.close()
        return out

    return run


def run_ragged(sims, out_dir: str, path: str = "tc_f16", group: int = 32, runner=None) -> list:
    """Run `sims` (phantoms.Workload objects) in groups of `group` simulations per
    simus_batch_rf call.  After every group, each simulation's RF [T][N][Nt] is saved to
    out_dir/rf_<index>.npy and the finished indices to out_dir/index.json (written
    atomically); simulations listed there are skipped.  Returns the indices run by this
    call.  `runner(list_of_workloads) -> list_of_arrays` replaces the GPU call in tests."""
    os.makedirs(out_dir, exist_ok=True)
    key = _key(sims)
    done = _load_index(out_dir, key)
    todo = [i for i in range(len(sims)) if i not in done or not os.path.exists(rf_path(out_dir, i))]
    run = runner or _gpu_runner(path)
    ran = []
    for g0 in range(0, len(todo), group):
        ids = todo[g0:g0 + group]
        outs = run([sims[i] for i in ids])
        for i, rf in zip(ids, outs):
            tmp = rf_path(out_dir, i) + ".tmp.npy"
            np.save(tmp, rf)
            os.replace(tmp, rf_path(out_dir, i))
        done.update(ids)
        _save_index(out_dir, key, done)
        ran.extend(ids)
    return ran
