"""Training state on disk (weights + Adam moments + step counter) for resume: round trip
and header validation (CPU)."""
import numpy as np
import pytest

from paper_2302_05170_b300 import pipeline
from paper_2302_05170_b300 import workloads as W


def test_round_trip(tmp_path):
    n = W.n_params(5, 7)
    rng = np.random.default_rng(0)
    P, am, av = (rng.normal(size=n).astype(np.float32) for _ in range(3))
    f = tmp_path / "state.npz"
    pipeline.save_training_state(f, P, am, av, 1234, 5, 7, act=1)
    st = pipeline.load_training_state(f)
    assert st["t"] == 1234 and st["d_in"] == 5 and st["m"] == 7 and st["act"] == 1
    for k, a in (("params", P), ("adam_m", am), ("adam_v", av)):
        assert np.array_equal(st[k], a)


def test_rejects_wrong_shapes(tmp_path):
    n = W.n_params(4, 7)
    with pytest.raises(ValueError):
        pipeline.save_training_state(tmp_path / "x.npz", np.zeros(n + 1), np.zeros(n), np.zeros(n), 0, 4, 7)
    f = tmp_path / "y.npz"
    np.savez(f, header=np.array([1, 4, 7, 50, 4, 0, 3]), params=np.zeros(n - 1, np.float32),
             adam_m=np.zeros(n, np.float32), adam_v=np.zeros(n, np.float32))
    with pytest.raises(ValueError):
        pipeline.load_training_state(f)
    g = tmp_path / "z.npz"
    np.savez(g, header=np.array([9, 4, 7, 50, 4, 0, 3]), params=np.zeros(n, np.float32),
             adam_m=np.zeros(n, np.float32), adam_v=np.zeros(n, np.float32))
    with pytest.raises(ValueError):
        pipeline.load_training_state(g)
