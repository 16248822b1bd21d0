"""Parity at the full sizes of the ragged batch and of the gradient workload, against the
FP64 oracle, through the C ABI.

Ragged batch (simulations of the seeded 256-simulation batch with 117,000 to 975,000
scatterers, 3 to 63 transmits, arrays of 68 to 174 elements): one
simus_batch_rf_spectrum launch, spectra compared with the oracle at 8 random bins per
simulation, every element and transmit.  The oracle's cost grows with S N T per bin, so
the four largest simulations keep one nonzero reflection coefficient per 128-scatterer
tile (at a random position in the tile) and zero elsewhere: a scatterer with R_s = 0
adds exactly nothing to Eq. 32, so the oracle is given the nonzero scatterers only,
while the GPU runs all of them through its tiles, chunks and work items.  A
simulation of 117,000 scatterers keeps every coefficient.

Gradient workload (128 elements, 11 plane waves, 10,000 scatterers): simus_rf_grad at
full size for a seeded upstream gradient; dL/dR, dL/dx and dL/dz at 24 sampled
scatterers against the oracle's adjoint.  The delay gradient is a sum over scatterers
for a fixed upstream gradient, so it is checked at full size by splitting the
scatterers into the sample A and the rest B: the GPU's full result equals its results
on A and on B added, and its result on A equals the oracle's.

Tolerances: 2e-3 relative L2 for the FP16 tensor-core contraction, 1e-5 for FP32.
"""
import numpy as np
import pytest
import torch

from paper_2102_02738_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu
TOL_TC, TOL_F32 = 2e-3, 1e-5
SPARSE = (210, 150, 207, 76)     # 805k, 798k, 974k, 940k scatterers
DENSE = (48,)                    # 117k scatterers, 154 elements (two receive halves)


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2102_02738_gb300 import build
    build.build()
    from paper_2102_02738_gb300 import simus
    return simus


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def one_per_tile(rc, seed):
    """Keep one coefficient per tile of 128 scatterers, at a seeded position."""
    n = rc.size
    tiles = (n + 127) // 128
    u = ph.uniform(seed, 21, tiles)
    keep = np.minimum(np.arange(tiles) * 128 + (u * 128).astype(np.int64), n - 1)
    out = np.zeros_like(rc)
    out[keep] = rc[keep]
    return out


def test_ragged_batch_large_simulations_sampled_bins(S, oracle):
    sims = ph.ragged_batch()            # the seeded 256-simulation batch
    picked = [sims[i] for i in SPARSE + DENSE]
    for i, w in zip(SPARSE, picked):
        w.rc = one_per_tile(w.rc, 3000 + i)
    plans = [S.Plan(w.cfg, path="tc_f16") for w in picked]
    txs = [(dev(w.delays), dev(w.apod)) for w in picked]
    scs = [(dev(w.x), None, dev(w.z), dev(w.rc)) for w in picked]
    specs = [torch.empty((w.n_tx, w.cfg["n_elements"], p.n_bins, 2), device="cuda")
             for w, p in zip(picked, plans)]
    S.simus_batch_rf_spectrum([p.handle for p in plans], txs, scs, specs)
    S.simus_plan_check(plans[0].handle)
    for k, (w, p, sp) in enumerate(zip(picked, plans, specs)):
        got = torch.view_as_complex(sp).cpu().numpy()
        nb = p.n_bins
        ks = np.unique((ph.uniform(4000 + k, 1, 8) * nb).astype(np.int64))
        nz = np.flatnonzero(w.rc)
        ref = oracle.rf_spectrum(w.cfg, w.delays, w.apod, w.x[nz], None, w.z[nz], w.rc[nz],
                                 p.info["q_lo"] + ks)
        err = rel_l2(got[..., ks], ref)
        assert err <= TOL_TC, f"{w.name}: S={w.n_scat} N={w.cfg['n_elements']} T={w.n_tx} rel-L2 {err:.2e}"
    for p in plans:
        p.close()


def test_gradient_workload_full_size(S, oracle):
    w = ph.planewave_linear_128_grad()
    T, N, nt = w.n_tx, w.cfg["n_elements"], w.cfg["n_samples"]
    drf = ph.normal(1004, 31, T * N * nt).reshape(T, N, nt).astype(np.float32)
    plan = S.Plan(w.cfg, path="plain")
    d_drf = dev(drf)

    def grad(sel):
        g = plan.rf_grad(dev(w.delays), dev(w.apod), dev(w.x[sel]), None, dev(w.z[sel]),
                         dev(w.rc[sel]), d_drf)
        S.simus_plan_check(plan.handle)
        return {k: v.cpu().numpy() for k, v in g.items()}

    full = grad(np.arange(w.n_scat))
    A = np.linspace(0, w.n_scat - 1, 24).astype(np.int64)
    B = np.setdiff1d(np.arange(w.n_scat), A)
    gR, gx, gz, gd = oracle.rf_grad(w.cfg, w.delays, w.apod, w.x[A], None, w.z[A], w.rc[A],
                                    drf)
    for name, ref in (("rc", gR), ("x", gx), ("z", gz)):
        err = rel_l2(full[name][A], ref)
        assert err <= TOL_F32, f"dL/d{name} at 24 scatterers of the full workload: {err:.2e}"
    on_a, on_b = grad(A), grad(B)
    assert rel_l2(on_a["delays"], gd) <= TOL_F32
    assert rel_l2(on_a["delays"] + on_b["delays"], full["delays"]) <= TOL_F32
    plan.close()
