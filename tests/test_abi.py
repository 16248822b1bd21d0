"""C-ABI checks that need no GPU: the library builds, loads and exports every entry
point that include/simus.h declares, the ctypes structures match the header's layout,
and the host-only helpers follow their definitions."""
import ctypes as C
import math
import os
import re
import subprocess

import pytest

from paper_2102_02738_gb300 import phantoms as ph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "simus.h")


@pytest.fixture(scope="module")
def S():
    from paper_2102_02738_gb300 import build
    build.build()
    from paper_2102_02738_gb300 import simus
    return simus


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(simus_\w+)\s*\(", src)))


def test_header_declares_the_abi():
    names = declared_functions()
    for want in ("simus_plan_create", "simus_plan_destroy", "simus_rf", "simus_pfield",
                 "simus_rf_grad", "simus_batch_rf", "simus_last_error", "simus_default_nt"):
        assert want in names


def test_library_exports_every_declared_symbol(S):
    lib = C.CDLL(S._build.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches_header(S, tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "simus.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(simus_probe), sizeof(simus_medium), sizeof(simus_tx),
         sizeof(simus_scat), sizeof(simus_plan_info));
  printf("%zu %zu %zu %zu\n", offsetof(simus_probe, pitch), offsetof(simus_medium, pulse_cycles),
         offsetof(simus_tx, apod), offsetof(simus_plan_info, df));
  printf("%zu %zu %zu %zu\n", sizeof(simus_tuning), offsetof(simus_tuning, chunks),
         offsetof(simus_tuning, depth_order), offsetof(simus_tuning, tensor_idft));
  return 0; }
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [C.sizeof(S.Probe), C.sizeof(S.Medium), C.sizeof(S.Tx), C.sizeof(S.Scat),
           C.sizeof(S.PlanInfo), S.Probe.pitch.offset, S.Medium.pulse_cycles.offset,
           S.Tx.apod.offset, S.PlanInfo.df.offset, C.sizeof(S.Tuning), S.Tuning.chunks.offset,
           S.Tuning.depth_order.offset, S.Tuning.tensor_idft.offset]
    assert [int(v) for v in out] == got


def test_default_nt_rule(S):
    w = ph.planewave_linear_128(n_scat=10)
    cfg = w.cfg
    for r_max, tau in ((0.03, 0.0), (0.0591, 1.3e-6), (0.12, 2e-5)):
        nt = S.simus_default_nt(cfg, r_max, tau)
        n = math.ceil(cfg["fs"] * (2 * r_max / cfg["c"] + tau + 8 / cfg["fc"]))
        assert nt == n + (n & 1) and nt % 2 == 0


def test_pfield_nfreq_matches_oracle(S, oracle):
    w = ph.focused_linear_64()
    for r_max, tau in ((0.02, 0.0), (0.05, 3e-6)):
        assert S.simus_pfield_nfreq(w.cfg, r_max, tau) == oracle.pfield_nfreq(w.cfg, r_max, tau)


@pytest.mark.parametrize("bad", [dict(n_elements=0), dict(width=1e-3), dict(frac_bw=0.0),
                                 dict(c=-1.0), dict(pulse=7), dict(height=0.0)])
def test_invalid_arguments_are_rejected_on_host(S, bad):
    cfg = dict(ph.planewave_linear_128(n_scat=4).cfg)
    cfg.update(bad)
    with pytest.raises(S.SimusError) as ei:
        S.simus_default_nt(cfg, 0.05, 0.0)
    assert ei.value.code == -1
    assert S.lib.simus_last_error().decode()


def test_tuning_rejects_null_plan(S):
    t = S.Tuning()
    assert S.lib.simus_plan_set_tuning(None, t) == -1
    assert S.lib.simus_plan_get_tuning(None, t) == -1
