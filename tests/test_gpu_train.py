"""GPU training of the collocation network (Algorithm I step 1) against the
oracle, and what the trained network gains.

* FP32 forward pass and MSE parameter gradient vs the oracle's FP64
  back-propagation (itself pinned by finite differences and torch.autograd):
  within 1e-5 of the largest gradient entry.
* Adam: several GPU steps vs the oracle's Adam on the same minibatches.
* End to end: labels from em_collocation_labels (GBM), GPU training, loss
  falls; the trained network approaches the exact GBM collocation map; and the
  gain test: with the same normals, the trained 7L sampler's strong error
  against the exact GBM solution at dt = 0.125 is far below that of plain
  Euler-Maruyama with the same coarse step (the method without the network).
"""
import math

import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _params(d_in, m, seed):
    P = W.xavier_params(d_in, m, seed=seed)
    rng = np.random.default_rng(seed)
    o = 0
    for (fo, fi) in W.layer_shapes(d_in, m):
        o += fo * fi
        P[o:o + fo] = rng.uniform(-0.1, 0.1, fo).astype(np.float32)
        o += fo
    return P


@pytest.mark.parametrize("act", [0, 1])
def test_forward_and_grad(sl, orc, act):
    d_in, m, n = 4, 7, 1000
    P = _params(d_in, m, 3)
    rng = np.random.default_rng(0)
    f = rng.uniform(0, 2, (n, d_in)).astype(np.float32)
    y = rng.standard_normal((n, m)).astype(np.float32)
    rows = rng.permutation(n)[:777].astype(np.int32)
    net = sl.make_net(_dev(P), d_in, m, act=act)
    out = sl.mlp_forward(net, _dev(f)).cpu().numpy()
    want = orc.mlp_forward(P.astype(np.float64), f, d_in, m, act=act)
    assert np.abs(out - want).max() <= 1e-5 * (np.abs(want).max() + 1)
    loss, g = sl.mse_grad(net, _dev(f), _dev(y), _dev(rows, torch.int32))
    lo, go = orc.mse_grad(P.astype(np.float64), f, y, d_in, m, rows=rows, act=act)
    assert loss.item() == pytest.approx(lo, rel=1e-5)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-5 * np.abs(go).max()


def test_adam_steps(sl, orc):
    d_in, m, batch, nb = 4, 7, 1024, 5
    P = _params(d_in, m, 4)
    rng = np.random.default_rng(1)
    n = 3000
    f = rng.uniform(0, 2, (n, d_in)).astype(np.float32)
    y = rng.standard_normal((n, m)).astype(np.float32)
    rows = W.minibatch_rows(n, batch, nb, seed=2)
    Pd = _dev(P)
    am, av = torch.zeros_like(Pd), torch.zeros_like(Pd)
    losses = sl.train(Pd, d_in, m, am, av, 0, _dev(f), _dev(y), _dev(rows, torch.int32), batch).cpu().numpy()
    Po, amo, avo, lo = orc.train_adam(P.astype(np.float64), np.zeros(P.size), np.zeros(P.size), 0, f, y,
                                      rows, batch, d_in, m, lr=1e-3)
    assert np.allclose(losses, lo, rtol=1e-4)
    dP = Pd.cpu().numpy() - P
    dPo = Po - P
    # Adam normalises the step: entries whose gradient is tiny can move by up to
    # ~lr in either precision; the rest must agree to 1e-3 of the learning rate.
    _, g0 = orc.mse_grad(P.astype(np.float64), f, y, d_in, m, rows=rows[0])
    big = np.abs(g0) > 1e-3 * np.abs(g0).max()
    assert np.abs(dP - dPo)[big].max() <= 1e-3 * 1e-3 * nb
    assert np.abs(dP - dPo).max() <= 2e-3 * nb


def test_train_gbm_and_gain(sl, orc):
    """Labels -> training -> 7L sampling, all on the GPU (GBM, m = 7, dt = 0.125)."""
    d_in, m, dt = 4, 7, 0.125
    n_rows, n_paths = 1 << 14, 100_000
    th, yi, dts = W.gbm_training_rows(n_rows, seed=2, dt=dt)
    lab = sl.em_collocation_labels(0, _dev(th), _dev(yi), _dev(dts), n_paths, 100, m, 7)
    feats = _dev(np.concatenate([yi[:, None], dts[:, None], th], 1).astype(np.float32))
    P = _dev(W.xavier_params(d_in, m, seed=0))
    am, av = torch.zeros_like(P), torch.zeros_like(P)
    batch, nb = 1024, 20000
    rows = _dev(W.minibatch_rows(n_rows, batch, nb, seed=3), torch.int32)
    losses = sl.train(P, d_in, m, am, av, 0, feats, lab, rows, batch).cpu().numpy()
    assert losses[-200:].mean() < 0.05 * losses[:20].mean()
    # trained map vs the exact lognormal collocation map on a grid
    x, _, _ = sl.gauss_hermite(m)
    net = sl.make_net(P, d_in, m)
    gy, gmu, gsg = np.meshgrid(np.linspace(0.5, 2.0, 7), np.linspace(0.02, 0.18, 5), np.linspace(0.15, 0.45, 5))
    G = np.stack([gy.ravel(), np.full(gy.size, dt), gmu.ravel(), gsg.ravel()], 1).astype(np.float32)
    yh = sl.mlp_forward(net, _dev(G)).cpu().numpy()
    ex = G[:, :1] * np.exp((G[:, 2:3] - 0.5 * G[:, 3:4] ** 2) * dt + G[:, 3:4] * math.sqrt(dt) * x[None, :])
    assert np.abs(yh - ex).max() / G[:, 0].max() < 0.05
    # gain test on one theta of the online workload: strong error vs the exact solution
    mu, sg, T, n_steps, n = 0.1, 0.3, 2.0, 16, 4000
    off = W.offsets_from_counts([n])
    for prec in (sl.PREC_FP32, sl.PREC_BF16):
        netp = sl.make_net(P, d_in, m, prec=prec)
        yt = torch.empty(n, device="cuda")
        sl.seven_league_simulate_batched(0, netp, _dev([[mu, sg]]), _dev([1.0]), _dev(off, torch.int64), T,
                                         n_steps, m, 11, out_YT=yt)
        y7 = yt.cpu().numpy().astype(np.float64)
        sx = np.array([orc.normals(11, 0, 0, q, 0, n_steps).sum() for q in range(n)])
        exact7 = np.exp((mu - 0.5 * sg * sg) * T + sg * math.sqrt(dt) * sx)
        err7 = np.abs(y7 - exact7).mean()
        # coarse Euler-Maruyama, same step, its own normals (tag 1 stream of row 0)
        em = sl.em_terminal(0, _dev([[mu, sg]]), _dev([1.0]), _dev([T]), n, n_steps, 11).cpu().numpy()[0]
        sxe = np.array([orc.normals(11, 1, 0, q, 0, n_steps).sum() for q in range(n)])
        exact_em = np.exp((mu - 0.5 * sg * sg) * T + sg * math.sqrt(dt) * sxe)
        err_em = np.abs(em - exact_em).mean()
        print('gain', prec, err7, err_em)
        assert err7 < 0.25 * err_em, (prec, err7, err_em)
