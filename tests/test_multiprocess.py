"""The N-GPU replica path of bench.py on CPU: two gloo ranks run the process-group setup,
the barrier and the max-over-ranks reduction that bench.py uses around its timed region,
and the reference arm (rank 0 alone runs and prints; the other rank exits without work).
The RF path itself has no collective: with N GPUs every rank runs an independent replica.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
rank, ws, local = bench.dist_init()
bench.barrier(ws)
v = bench.allreduce_max(float(rank + 1) * 10.0, ws)
with open(os.path.join({out!r}, f"rank{{rank}}.json"), "w") as fh:   # no interleaved stdout
    json.dump({{"rank": rank, "ws": ws, "max": v}}, fh)
import torch.distributed as dist
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch(code, nproc, extra_args=()):
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), *code]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    return subprocess.run(cmd + list(extra_args), capture_output=True, text=True, timeout=300,
                          cwd=ROOT, env=env)


def test_gloo_barrier_and_max(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT, out=str(tmp_path)))
    r = launch([str(script)], 2)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in (0, 1)]
    assert sorted(d["rank"] for d in lines) == [0, 1]
    assert all(d["ws"] == 2 and d["max"] == 20.0 for d in lines)


@pytest.mark.slow
def test_reference_arm_two_ranks():
    r = launch(["bench.py", "--impl", "reference", "--workload", "focused-linear-64",
                "--gpus", "2", "--steps", "1", "--warmup", "0"], 2)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1                      # rank 0 alone prints
    line = lines[0]
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
