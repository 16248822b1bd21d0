"""The tensor-core path's tuning interface and the autotuner.

Tunings change launch shapes only: every candidate must give the same RF as the FP64
oracle within the tensor-core tolerance (2e-3 relative L2), and the direct and tabulated
delta must agree to the table's error.  The autotuner must pick one of the timed
candidates, set it on the plan and cache it under the problem's shape key.
"""
import json

import numpy as np
import pytest
import torch

from paper_2102_02738_gb300 import phantoms as ph

TOL_TC = 2e-3


def test_candidates_cover_the_knobs():
    from paper_2102_02738_gb300 import autotune
    c = autotune.candidates(single=True)
    assert {k for d in c for k in d} == {"max_bins", "pair", "delta_table", "chunks", "tile_buffers"}
    assert {d["pair"] for d in c} == {0, 1, 2} and {d["delta_table"] for d in c} == {0, 1}
    assert {d["tile_buffers"] for d in c if d["pair"] > 0} == {1, 2}
    cb = autotune.candidates(single=False)
    assert {d["items_per_sm"] for d in cb} == {2, 4, 8}
    assert {d["max_bins"] for d in c} == {2, 3, 4, 6}
    assert autotune._bucket(1) == 1 and autotune._bucket(1000) == 1024 and autotune._bucket(1024) == 1024


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


@pytest.mark.gpu
def test_set_get_round_trip(S):
    w = ph.tiny(n_elements=16, n_scat=50, n_tx=3)
    plan = S.Plan(w.cfg, path="tc_f16")
    default = dict(items_per_sm=4, max_bins=4, pair=2, delta_table=1, chunks=0, tile_buffers=2,
                   depth_order=1, tensor_idft=1)
    assert plan.get_tuning() == default
    plan.set_tuning(max_bins=6, pair=0, delta_table=0, chunks=3, items_per_sm=8, tile_buffers=1,
                    depth_order=0, tensor_idft=0)
    assert plan.get_tuning() == dict(items_per_sm=8, max_bins=6, pair=0, delta_table=0, chunks=3,
                                     tile_buffers=1, depth_order=0, tensor_idft=0)
    plan.set_tuning(max_bins=-1, pair=-1, delta_table=-1, chunks=0, items_per_sm=-1, tile_buffers=0,
                    depth_order=-1, tensor_idft=-1)
    assert plan.get_tuning() == default
    with pytest.raises(S.SimusError):
        plan.set_tuning(max_bins=65)
    with pytest.raises(S.SimusError):
        plan.set_tuning(pair=3)
    with pytest.raises(S.SimusError):
        plan.set_tuning(tile_buffers=3)
    with pytest.raises(S.SimusError):
        plan.set_tuning(depth_order=2)
    with pytest.raises(S.SimusError):
        plan.set_tuning(tensor_idft=2)
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("convex", [False, True])
def test_depth_order_matches_the_given_order_and_the_oracle(S, oracle, convex):
    """Scatterers copied in distance-to-array order before the launch: the RF matches the
    caller's order and the FP64 oracle within the tensor-core tolerance, and two calls in a
    row give the same bits (the stable sort puts every scatterer at the same place)."""
    w = ph.tiny(convex=convex, n_elements=24, n_scat=900, n_tx=5, nt=500)
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    plan = S.Plan(w.cfg, path="tc_f16")
    args = [dev(v) for v in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    a = plan.rf(*args).cpu().numpy()
    b = plan.rf(*args).cpu().numpy()
    plan.set_tuning(depth_order=0)
    c = plan.rf(*args).cpu().numpy()
    plan.close()
    assert np.array_equal(a, b)
    assert rel_l2(a, ref) <= 2e-3
    assert rel_l2(c, ref) <= 2e-3
    assert rel_l2(a, c) <= 2e-3


@pytest.mark.gpu
@pytest.mark.parametrize("case", [
    dict(n_elements=24, n_tx=5, nt=500, path="tc_f16"),       # 120 channels: one ragged tile
    dict(n_elements=64, n_tx=5, nt=700, path="tc_bf16"),      # 320 channels: two tiles, ragged
    dict(n_elements=16, n_tx=3, nt=96, path="tc_f16"),        # fewer K chunks than stages
    dict(n_elements=48, n_tx=11, nt=1031, path="tc_f16"),     # 528 channels, nt ragged by 7
])
def test_tensor_idft_matches_the_cuda_core_idft(S, oracle, case):
    """The inverse DFT on the tensor cores (split-BF16 twiddles and spectra, FP32
    accumulation, about 2^-16 relative per term) against the FP32 CUDA-core iDFT of the
    same spectrum, over channel and sample counts that leave ragged tiles, and both
    against the FP64 oracle."""
    w = ph.tiny(convex=True, n_elements=case["n_elements"], n_scat=300, n_tx=case["n_tx"],
                nt=case["nt"])
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    plan = S.Plan(w.cfg, path=case["path"])
    args = [dev(v) for v in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    a = plan.rf(*args).cpu().numpy()
    b = plan.rf(*args).cpu().numpy()
    plan.set_tuning(tensor_idft=0)
    c = plan.rf(*args).cpu().numpy()
    assert S.lib.simus_plan_check(plan.handle) == 0
    plan.close()
    assert a.shape == c.shape == ref.shape
    assert np.array_equal(a, b)
    assert rel_l2(a, c) <= 1e-4
    assert float(np.abs(a - c).max()) <= 1e-4 * float(np.abs(c).max())
    assert rel_l2(a, ref) <= TOL_TC


@pytest.mark.gpu
def test_tensor_idft_launches_its_own_kernels(S):
    """With tensor_idft = 1 the iDFT stage is two launches of this library (the spectra
    blocked into split BF16, then the tcgen05 product), with 0 one (the CUDA-core iDFT);
    nothing else in the call changes."""
    w = ph.tiny(convex=True, n_elements=16, n_scat=100, n_tx=3, nt=300)
    plan = S.Plan(w.cfg, path="tc_f16")
    args = [dev(v) for v in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    plan.rf(*args)                                   # warm-up: workspace, staging
    counts = []
    for t in (1, 0):
        plan.set_tuning(tensor_idft=t)
        torch.cuda.synchronize()
        n0 = S.simus_kernel_launches()
        plan.rf(*args)
        torch.cuda.synchronize()
        counts.append(S.simus_kernel_launches() - n0)
    assert S.lib.simus_plan_check(plan.handle) == 0
    plan.close()
    assert counts[0] == counts[1] + 1


@pytest.mark.gpu
@pytest.mark.parametrize("tun", [dict(max_bins=2, pair=1, delta_table=1),
                                 dict(max_bins=6, pair=2, delta_table=1),
                                 dict(max_bins=3, pair=2, delta_table=0, chunks=3),
                                 dict(max_bins=6, pair=1, delta_table=0, chunks=2),
                                 dict(max_bins=3, pair=0, delta_table=1, chunks=1),
                                 dict(max_bins=8, pair=0, delta_table=0),
                                 dict(max_bins=6, pair=2, delta_table=1, tile_buffers=1),
                                 dict(max_bins=4, pair=1, delta_table=0, tile_buffers=1)])
def test_every_tuning_matches_the_oracle(S, oracle, tun):
    w = ph.tiny(convex=True, n_elements=24, n_scat=400, n_tx=9)
    ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
    plan = S.Plan(w.cfg, path="tc_f16")
    plan.set_tuning(**tun)
    got = plan.rf(*[dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]).cpu().numpy()
    assert S.lib.simus_plan_check(plan.handle) == 0
    plan.close()
    assert rel_l2(got, ref) <= TOL_TC


@pytest.mark.gpu
def test_delta_table_agrees_with_direct_evaluation(S):
    # same FP16 operands up to the error of the table's quadratic pieces (1.9e-5 relative
    # inside an interval, at most 3e-4 half an interval beyond it): below FP16 rounding
    w = ph.tiny(convex=True, n_elements=32, n_scat=600, n_tx=5)
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    outs = []
    for tab in (1, 0):
        plan = S.Plan(w.cfg, path="tc_f16")
        plan.set_tuning(delta_table=tab)
        outs.append(plan.rf(*args).cpu().numpy())
        plan.close()
    assert rel_l2(outs[0], outs[1]) <= 2e-4


@pytest.mark.gpu
def test_autotuner_picks_and_caches(S, tmp_path):
    from paper_2102_02738_gb300 import autotune
    w = ph.tiny(n_elements=32, n_scat=700, n_tx=4)
    args = [dev(a) for a in (w.delays, w.apod, w.x, w.y, w.z, w.rc)]
    plan = S.Plan(w.cfg, path="tc_f16")
    cache = tmp_path / "tune.json"
    cands = [dict(max_bins=2, pair=1, delta_table=1, chunks=0), dict(max_bins=4, pair=0, delta_table=0, chunks=0)]
    r = autotune.tune_rf(plan, *args, reps=1, cache_path=str(cache), cands=cands)
    assert r["best"] in cands and len(r["all"]) == 2 and r["ms"] > 0
    assert plan.get_tuning()["max_bins"] == r["best"]["max_bins"]
    key = autotune.shape_key(plan, w.n_tx, w.n_scat)
    assert key in json.loads(cache.read_text())
    plan2 = S.Plan(w.cfg, path="tc_f16")
    assert autotune.apply_cached(plan2, w.n_tx, w.n_scat, cache_path=str(cache))
    assert plan2.get_tuning()["pair"] == r["best"]["pair"]
    plan.close()
    plan2.close()
