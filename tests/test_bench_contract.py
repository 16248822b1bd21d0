"""bench.py's contract, on the CPU: the ALU roofline denominator and the reference arm's
JSON line (the FP64 oracle timed on the host cores, one line with the keys the
benchmark's consumers read)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_alu_peak_is_the_sfu_bound_of_the_term_budget():
    import bench
    # 85 FP32-pipe + 12 SFU instructions per unique term; 128 FP32 and 16 SFU lanes per SM
    fp32 = 152 * 128 * 2070e6 / 85
    sfu = 152 * 16 * 2070e6 / 12
    assert sfu < fp32
    assert bench.alu_peak_terms(152, 2070.0) == pytest.approx(sfu, rel=1e-12)
    assert bench.alu_peak_terms(152, 2070.0) == pytest.approx(4.1952e11, rel=1e-4)
    assert bench.alu_peak_terms(76, 2070.0) == pytest.approx(sfu / 2, rel=1e-12)


def test_every_workload_has_a_generator():
    import bench
    from paper_2102_02738_gb300 import phantoms as ph
    assert bench.DEFAULT_WORKLOAD in bench.WORKLOADS
    for name, fn in bench.WORKLOADS.items():
        assert callable(fn) and fn.__module__ == ph.__name__, name


def test_reference_arm_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                        "focused-linear-64", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "focused-linear-64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]
    # the same config dict as the GPU arm prints for this workload
    import bench
    from oracle import oracle
    from paper_2102_02738_gb300 import phantoms as ph
    w = ph.focused_linear_64()
    lo, hi, nb = oracle.bins(w.cfg)
    assert d["config"] == json.loads(json.dumps(bench.workload_config("focused-linear-64", w, nb,
                                                                      oracle.nsub(w.cfg))))
