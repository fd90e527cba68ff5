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


@pytest.mark.parametrize("act", [0, 1])
def test_fold_normalization(orc, act):
    """A network trained on normalised features and labels, folded into its first and last
    layers, maps the raw features to the raw labels: against the oracle's forward pass of the
    unfolded network on the normalised features, de-normalised (FP64)."""
    import torch
    d_in, m = 4, 7
    P = W.xavier_params(d_in, m, seed=7)
    rng = np.random.default_rng(3)
    f = np.stack([rng.uniform(0.25, 4, 200), rng.choice([0.125, 0.5], 200), rng.uniform(0, 0.2, 200),
                  rng.uniform(0.1, 0.5, 200)], 1)
    fsh, fsc = f.mean(0), f.std(0)
    ysh, ysc = rng.uniform(0.5, 2, m), rng.uniform(0.1, 1, m)
    Pf = pipeline.fold_normalization(torch.as_tensor(P), d_in, m, fsh, fsc, ysh, ysc).numpy()
    want = orc.mlp_forward(P.astype(np.float64), (f - fsh) / fsc, d_in, m, act=act) * ysc + ysh
    got = orc.mlp_forward(Pf.astype(np.float64), f, d_in, m, act=act)
    assert np.allclose(got, want, rtol=1e-5, atol=1e-5 * np.abs(want).max())
    # every layer but the first and the last is untouched
    o1 = 50 * d_in + 50
    o5 = W.n_params(d_in, m) - (m * 50 + m)
    assert np.array_equal(Pf[o1:o5], P[o1:o5])
