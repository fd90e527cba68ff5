"""GPU training of the collocation network (Algorithm I step 1) against the
oracle, and what the trained network gains.

* FP32 forward pass and MSE parameter gradient vs the oracle's FP64
  back-propagation (itself pinned by finite differences and torch.autograd):
  within 1e-5 of the largest gradient entry.
* BF16-aware gradient (net->prec = BF16): the oracle's gradient of the network with
  BF16-rounded weights and biases, within the same 1e-5; the BF16-finished pipeline
  returns BF16-valued weights, and with them the two sampler forms agree path by path
  within the BF16 gate.
* Adam: several GPU steps vs the oracle's Adam on the same minibatches.
* End to end: labels from em_collocation_labels (GBM), GPU training (normalised
  features and labels, then a BF16 finish), loss falls; the trained network
  approaches the exact GBM collocation map; and the gain test, each method driven
  by its own normals against the exact GBM solution: Euler-Maruyama's strong
  error grows as the coarse step grows (dt = 0.125 -> 1) while the trained 7L
  scheme's does not, and at dt = 1 the 7L strong error is below 0.4 of
  Euler-Maruyama's.  (The call prices of 4000 paths are printed, not compared:
  their standard error, ~0.007, is as large as either method's bias.  At
  dt = 0.125 the trained network is not more accurate per path than
  Euler-Maruyama: the paper's claim concerns large steps.)  Both forms of the
  sampler run the same BF16-valued trained network, and their errors agree.
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


@pytest.mark.parametrize("act", [0, 1])
def test_bf16_aware_grad(sl, orc, act):
    d_in, m, n = 4, 7, 1000
    P = _params(d_in, m, 6) * np.float32(1.37)                 # not BF16 values: rounding matters
    rng = np.random.default_rng(2)
    f = rng.uniform(0, 2, (n, d_in)).astype(np.float32)
    y = rng.standard_normal((n, m)).astype(np.float32)
    net = sl.make_net(_dev(P), d_in, m, act=act, prec=sl.PREC_BF16)
    loss, g = sl.mse_grad(net, _dev(f), _dev(y))
    Pb = W.bf16_round(P).astype(np.float64)
    lo, go = orc.mse_grad(Pb, f, y, d_in, m, act=act)
    assert loss.item() == pytest.approx(lo, rel=1e-5)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-5 * np.abs(go).max()
    lo32, go32 = orc.mse_grad(P.astype(np.float64), f, y, d_in, m, act=act)
    assert np.abs(go32 - go).max() > 1e-3 * np.abs(go).max()   # and it is not the FP32 network's


def test_bf16_finished_network_runs_alike_in_both_forms(sl, orc):
    """pipeline.train_network with a BF16 finish: every weight is a BF16 value, and the FP32 and
    tensor-core forms of the sampler on it agree path by path (gate 2e-3, 16 steps)."""
    from paper_2302_05170_b300 import pipeline
    th, yi, dt = W.gbm_training_rows(4096, seed=4)
    P, losses, _ = pipeline.train_network(0, th, yi, dt, 7, n_paths=20000, n_steps=4000, normalize=True,
                                          bf16_steps=1000)
    assert torch.equal(P, P.to(torch.bfloat16).float())
    w = W.gbm_online(n_paths_per_set=20000)
    ths, y0, off = _dev(w["theta"]), _dev(w["Y0"]), _dev(w["offsets"], torch.int64)
    out = []
    for prec in (sl.PREC_FP32, sl.PREC_BF16):
        yt = torch.empty(int(w["offsets"][-1]), device="cuda")
        sl.seven_league_simulate_batched(0, sl.make_net(P, 4, 7, prec=prec), ths, y0, off, 2.0, 16, 7, 1, out_YT=yt)
        out.append(yt.cpu().numpy().astype(np.float64))
    err = rel_err(out[1], out[0], 1.0)
    print("BF16 vs FP32 form on the same BF16 weights: max %.3g, p99.99 %.3g" % (err.max(), np.percentile(err, 99.99)))
    assert np.percentile(err, 99.99) <= 2e-3


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


def _strong_errors(sl, orc, P, n_steps, n=4000, mu=0.1, sg=0.3, T=2.0, m=7, seed=11):
    """Mean |Y_T - exact| for the trained 7L sampler (FP32 and BF16 forms), the
    exact-collocation 7L sampler, and Euler-Maruyama with the same coarse step, each
    against the exact GBM solution driven by that method's own normals; plus the
    call price E[(Y_T - 1)+] of each method."""
    dt = T / n_steps
    off = W.offsets_from_counts([n])
    th, y0, offd = _dev([[mu, sg]]), _dev([1.0]), _dev(off, torch.int64)
    sx = np.array([orc.normals(seed, 0, 0, q, 0, n_steps).sum() for q in range(n)])
    exact7 = np.exp((mu - 0.5 * sg * sg) * T + sg * math.sqrt(dt) * sx)
    out = {}
    for name, model, net in (("fp32", 0, sl.make_net(P, 4, m, prec=sl.PREC_FP32)),
                             ("bf16", 0, sl.make_net(P, 4, m, prec=sl.PREC_BF16)),
                             ("exact", 1, None)):
        yt = torch.empty(n, device="cuda")
        sl.seven_league_simulate_batched(model, net, th, y0, offd, T, n_steps, m, seed, out_YT=yt)
        y = yt.cpu().numpy().astype(np.float64)
        out[name] = (np.abs(y - exact7).mean(), np.maximum(y - 1, 0).mean())
    em = sl.em_terminal(0, th, y0, _dev([T]), n, n_steps, seed).cpu().numpy()[0].astype(np.float64)
    sxe = np.array([orc.normals(seed, 1, 0, q, 0, n_steps).sum() for q in range(n)])
    exact_em = np.exp((mu - 0.5 * sg * sg) * T + sg * math.sqrt(dt) * sxe)
    out["em"] = (np.abs(em - exact_em).mean(), np.maximum(em - 1, 0).mean())
    return out


def test_train_gbm_and_gain(sl, orc):
    """Labels -> training -> 7L sampling, all on the GPU (GBM, m = 7), and the gain
    over plain Euler-Maruyama: the 7L error does not grow with the step size (the
    paper's claim) while Euler-Maruyama's does."""
    from paper_2302_05170_b300 import pipeline
    P, losses, lab = pipeline.train_gbm_online_network(n_rows=1 << 14, n_steps=40000, normalize=True,
                                                       n_paths=400_000, bf16_steps=10_000)
    assert losses[-500:].mean() < 0.02 * losses[:20].mean()
    assert torch.equal(P, P.to(torch.bfloat16).float())          # the BF16 network is the trained one
    d_in, m = 4, 7
    # trained map vs the exact lognormal collocation map on a grid (dt = 0.5)
    x, _, _ = sl.gauss_hermite(m)
    net = sl.make_net(P, d_in, m)
    gy, gmu, gsg = np.meshgrid(np.linspace(0.5, 2.0, 7), np.linspace(0.02, 0.18, 5), np.linspace(0.15, 0.45, 5))
    G = np.stack([gy.ravel(), np.full(gy.size, 0.5), gmu.ravel(), gsg.ravel()], 1).astype(np.float32)
    yh = sl.mlp_forward(net, _dev(G)).cpu().numpy()
    ex = G[:, :1] * np.exp((G[:, 2:3] - 0.5 * G[:, 3:4] ** 2) * 0.5 + G[:, 3:4] * math.sqrt(0.5) * x[None, :])
    print("max |H - exact map| / max Y on the grid:", np.abs(yh - ex).max() / G[:, 0].max())
    assert np.abs(yh - ex).max() / G[:, 0].max() < 0.1
    errs = {k: _strong_errors(sl, orc, P, k) for k in (16, 4, 2)}
    print("strong / call-price errors by number of steps:", errs)
    bs = math.exp(0.2) * stats_norm_cdf((0.2 + 0.045 * 2) / (0.3 * math.sqrt(2))) - \
        stats_norm_cdf((0.2 - 0.045 * 2) / (0.3 * math.sqrt(2)))
    # Euler-Maruyama degrades with the step; the trained 7L scheme does not, in either network form
    # (both run the same BF16-valued weights: their errors agree to the BF16 activations' rounding)
    assert errs[2]["em"][0] > 2.0 * errs[16]["em"][0]
    for form in ("fp32", "bf16"):
        assert errs[2][form][0] <= errs[16][form][0], form
        # gain at the largest step (dt = 1) in the strong error and in the call price
        assert errs[2][form][0] < 0.4 * errs[2]["em"][0], form
    for k in (16, 4, 2):
        assert errs[k]["bf16"][0] == pytest.approx(errs[k]["fp32"][0], rel=1e-2)
    for k in (16, 4, 2):   # the exact collocation map is far better than either trained form
        assert errs[k]["exact"][0] < 0.2 * min(errs[k]["fp32"][0], errs[k]["bf16"][0])


def stats_norm_cdf(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def test_resume_from_saved_state(sl, orc, tmp_path):
    """Training 2 x 50 Adam steps with a save/load of (weights, moments, step) in between gives
    bit-identical weights to 100 uninterrupted steps (Adam and the minibatch order are
    deterministic)."""
    from paper_2302_05170_b300 import pipeline
    th, yi, dt = W.gbm_training_rows(512, seed=9)
    feats = torch.as_tensor(np.concatenate([yi[:, None], dt[:, None], th], 1).astype(np.float32), device="cuda")
    labels = torch.as_tensor(np.random.default_rng(1).normal(1.0, 0.2, (512, 7)).astype(np.float32), device="cuda")
    rows = torch.as_tensor(W.minibatch_rows(512, 128, 100, seed=2), device="cuda")
    P0 = torch.as_tensor(W.xavier_params(4, 7, seed=0), device="cuda")

    P, am, av = P0.clone(), torch.zeros_like(P0), torch.zeros_like(P0)
    sl.train(P, 4, 7, am, av, 0, feats, labels, rows, 128, lr=1e-3)
    straight = P.cpu().numpy()

    P, am, av = P0.clone(), torch.zeros_like(P0), torch.zeros_like(P0)
    sl.train(P, 4, 7, am, av, 0, feats, labels, rows[:50], 128, lr=1e-3)
    pipeline.save_training_state(tmp_path / "s.npz", P, am, av, 50, 4, 7)
    st = pipeline.load_training_state(tmp_path / "s.npz", device="cuda")
    P, am, av = st["params"], st["adam_m"], st["adam_v"]
    sl.train(P, 4, 7, am, av, st["t"], feats, labels, rows[50:], 128, lr=1e-3)
    assert np.array_equal(P.cpu().numpy(), straight)
