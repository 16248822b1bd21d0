"""Ragged batches (simus_batch_rf: one persistent tensor-core launch over the work items
of every simulation) and the tensor-core kernel's general shapes (N > 128 elements in
two receive halves, transmits split into groups), against the FP64 oracle through the
C ABI.  Also: a batch captured in a CUDA graph replays to the same result.

Tolerances: 2e-3 relative L2 for the FP16 tensor-core path, 1e-5 for the FP32 path.
"""
import numpy as np
import pytest
import torch

from paper_2102_02738_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu
TOL_TC, TOL_F32 = 2e-3, 1e-5


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


def oracle_rf(oracle, w):
    return oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)


def single(S, w, path):
    plan = S.Plan(w.cfg, path=path)
    out = plan.rf(*[dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)])
    S.simus_plan_check(plan.handle)
    plan.close()
    return out.cpu().numpy()


@pytest.mark.parametrize("kw", [
    dict(n_elements=150, n_sub=1, n_scat=140, n_tx=3, nt=500),     # two receive halves
    dict(n_elements=192, n_sub=1, n_scat=130, n_tx=75, nt=420),    # + transmit groups
    dict(n_elements=40, n_sub=2, n_scat=260, n_tx=70, nt=420),     # wide transmit group
])
def test_tc_general_shapes(S, oracle, kw):
    w = ph.tiny(**kw)
    assert rel_l2(single(S, w, "tc_f16"), oracle_rf(oracle, w)) <= TOL_TC


@pytest.mark.parametrize("kw", [
    dict(n_elements=150, n_sub=1, n_scat=140, n_tx=3, nt=500),     # rows of two 128-element chunks
    dict(n_elements=192, n_sub=2, n_scat=130, n_tx=5, nt=420),
])
def test_plain_multi_transmit_wide_arrays(S, oracle, kw):
    # the multi-transmit FP32 kernel accumulates RF over elements 32 apart in chunks of 128
    w = ph.tiny(**kw)
    assert rel_l2(single(S, w, "plain"), oracle_rf(oracle, w)) <= TOL_F32


def ragged(n_sims=6, scale=1.0, seed=1005):
    sims = ph.ragged_batch(seed=seed, n_sims=n_sims, s_min=200, s_max=3000, scale=scale)
    for w in sims:   # keep the oracle fast: short RF records
        w.cfg["n_samples"] = min(w.cfg["n_samples"], 700)
    return sims


def run_batch(S, sims, path, stream=None):
    plans = [S.Plan(w.cfg, path=path) for w in sims]
    txs = [(dev(w.delays), dev(w.apod)) for w in sims]
    scs = [(dev(w.x), None, dev(w.z), dev(w.rc)) for w in sims]
    rfs = [torch.empty((w.n_tx, w.cfg["n_elements"], w.cfg["n_samples"]), device="cuda") for w in sims]
    S.simus_batch_rf([p.handle for p in plans], txs, scs, rfs, stream)
    return plans, txs, scs, rfs


def test_ragged_batch_tc_matches_oracle(S, oracle):
    sims = ragged()
    plans, _, _, rfs = run_batch(S, sims, "tc_f16")
    S.simus_plan_check(plans[0].handle)
    for w, rf in zip(sims, rfs):
        assert rel_l2(rf.cpu().numpy(), oracle_rf(oracle, w)) <= TOL_TC, w.name


def test_ragged_batch_bf16_matches_oracle(S, oracle):
    sims = [w for w in ragged(n_sims=10, seed=1006) if w.cfg["n_elements"] <= 176][:5]
    plans, _, _, rfs = run_batch(S, sims, "tc_bf16")
    S.simus_plan_check(plans[0].handle)
    for w, rf in zip(sims, rfs):
        assert rel_l2(rf.cpu().numpy(), oracle_rf(oracle, w)) <= TOL_TC, w.name


def test_ragged_batch_plain_matches_oracle(S, oracle):
    sims = ragged(n_sims=3)
    _, _, _, rfs = run_batch(S, sims, "plain")
    for w, rf in zip(sims, rfs):
        assert rel_l2(rf.cpu().numpy(), oracle_rf(oracle, w)) <= TOL_F32, w.name


@pytest.mark.parametrize("path,tol", [("plain", TOL_F32), ("tc_f16", TOL_TC)])
def test_batch_spectrum_matches_single_calls_and_oracle(S, oracle, path, tol):
    """simus_batch_rf_spectrum returns each simulation's spectrum before the inverse DFT:
    the same as simus_rf_spectrum on its own plan (up to the work split's summation order)
    and the oracle's at every kept bin."""
    sims = ragged(n_sims=3, seed=1007)
    plans = [S.Plan(w.cfg, path=path) for w in sims]
    txs = [(dev(w.delays), dev(w.apod)) for w in sims]
    scs = [(dev(w.x), None, dev(w.z), dev(w.rc)) for w in sims]
    specs = [torch.empty((w.n_tx, w.cfg["n_elements"], p.n_bins, 2), device="cuda")
             for w, p in zip(sims, plans)]
    S.simus_batch_rf_spectrum([p.handle for p in plans], txs, scs, specs)
    S.simus_plan_check(plans[0].handle)
    for w, p, sp, tx, sc in zip(sims, plans, specs, txs, scs):
        got = torch.view_as_complex(sp).cpu().numpy()
        one = p.rf_spectrum(*tx, *sc).cpu().numpy()
        qs = np.arange(p.info["q_lo"], p.info["q_hi"] + 1)
        ref = oracle.rf_spectrum(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc, qs)
        assert rel_l2(got, one) <= tol, w.name
        assert rel_l2(got, ref) <= tol, w.name
    for p in plans:
        p.close()


def test_batch_with_an_empty_simulation(S):
    sims = ragged(n_sims=3)
    sims[1].x, sims[1].z, sims[1].rc = (np.zeros(0, np.float32),) * 3
    _, _, _, rfs = run_batch(S, sims, "tc_f16")
    torch.cuda.synchronize()
    assert torch.count_nonzero(rfs[1]).item() == 0
    assert torch.count_nonzero(rfs[0]).item() > 0


@pytest.mark.parametrize("path", ["tc_f16", "tc_bf16"])
def test_batch_graph_replay(S, path):
    """The whole batch call is stream-capturable (after a warm-up call has sized the
    workspace and the staging buffer): replaying the graph reproduces the eager result."""
    sims = [w for w in ragged(n_sims=6, seed=77) if w.cfg["n_elements"] <= 176][:4]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plans, txs, scs, rfs = run_batch(S, sims, path, stream=st)
    st.synchronize()
    eager = [r.clone() for r in rfs]
    for r in rfs:
        r.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        S.simus_batch_rf([p.handle for p in plans], txs, scs, rfs, st)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, rfs):
        assert torch.equal(a, b)
