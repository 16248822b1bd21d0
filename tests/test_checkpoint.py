"""Checkpointed ragged batches: finished simulations are skipped on a rerun, an
interrupted run resumes where it stopped, a directory of another batch is refused, and
(on the GPU) the saved RF matches the FP64 oracle."""
import numpy as np
import pytest

from paper_2102_02738_gb300 import batch
from paper_2102_02738_gb300 import phantoms as ph


def sims(n=5):
    return [ph.tiny(seed=20 + i, n_elements=4 + i, n_scat=3 + i, n_tx=1 + i % 2) for i in range(n)]


class Fake:
    """Stands in for the GPU: returns a deterministic array per simulation."""

    def __init__(self, fail_after=None):
        self.calls, self.fail_after = [], fail_after

    def __call__(self, group):
        if self.fail_after is not None and len(self.calls) >= self.fail_after:
            raise RuntimeError("interrupted")
        self.calls.append([w.cfg["n_elements"] for w in group])
        return [np.full((w.n_tx, w.cfg["n_elements"], 8), float(w.cfg["n_elements"]), np.float32)
                for w in group]


def test_rerun_skips_finished(tmp_path):
    s = sims()
    f = Fake()
    assert batch.run_ragged(s, str(tmp_path), group=2, runner=f) == [0, 1, 2, 3, 4]
    assert len(f.calls) == 3
    g = Fake()
    assert batch.run_ragged(s, str(tmp_path), group=2, runner=g) == []
    assert g.calls == []
    for i, w in enumerate(s):
        assert np.load(batch.rf_path(str(tmp_path), i))[0, 0, 0] == w.cfg["n_elements"]


def test_interrupted_run_resumes(tmp_path):
    s = sims()
    f = Fake(fail_after=1)
    with pytest.raises(RuntimeError):
        batch.run_ragged(s, str(tmp_path), group=2, runner=f)
    g = Fake()
    assert batch.run_ragged(s, str(tmp_path), group=2, runner=g) == [2, 3, 4]
    assert g.calls == [[6, 7], [8]]


def test_missing_file_is_rerun(tmp_path):
    s = sims(3)
    batch.run_ragged(s, str(tmp_path), group=3, runner=Fake())
    (tmp_path / "rf_00001.npy").unlink()
    assert batch.run_ragged(s, str(tmp_path), group=3, runner=Fake()) == [1]


def test_other_batch_is_refused(tmp_path):
    batch.run_ragged(sims(3), str(tmp_path), runner=Fake())
    with pytest.raises(ValueError):
        batch.run_ragged(sims(4), str(tmp_path), runner=Fake())


@pytest.mark.gpu
def test_gpu_batch_checkpoint_matches_oracle(tmp_path, oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2102_02738_gb300 import build
    build.build()
    s = [ph.tiny(seed=30 + i, n_elements=8 + 4 * i, n_scat=60, n_tx=2) for i in range(3)]
    assert batch.run_ragged(s, str(tmp_path), group=2) == [0, 1, 2]
    for i, w in enumerate(s):
        ref = oracle.rf(w.cfg, w.delays, w.apod, w.x, w.y, w.z, w.rc)
        got = np.load(batch.rf_path(str(tmp_path), i))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-3
    assert batch.run_ragged(s, str(tmp_path), group=2) == []
