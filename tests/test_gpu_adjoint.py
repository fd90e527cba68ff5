"""GPU parity of the adjoint (pathwise sensitivities of E[max(Y_T - K, 0)]).

* Per path: reverse-mode GPU sensitivities (FP32) against the oracle's
  forward-mode propagation (FP64) on the same paths, for the exact GBM and
  OU maps and for networks with ReLU and Softplus; paths within 1e-4 of the
  kink (Y_T = K) are excluded because the two precisions may put them on
  different sides of it.
* Checkpoint interval: k = 1, 3, 8, 16 and n_steps give bit-identical results.
* Per-set means: FP64 means of the per-path values; seed_grad scales them.
* Central finite differences of the oracle's FP64 path mean (common random
  numbers) agree within 1e-3 relative.
* Exact GBM (m = 7, dt = 1/64) against closed-form Black-Scholes price,
  delta, vega and d/dmu within Monte Carlo error.
* torch.autograd through the SevenLeagueCall function.
"""
import math

import numpy as np
import pytest
import torch
from scipy import stats

from paper_2302_05170_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _adj(sl, model, net, th, y0, off, T, n_steps, m, seed, K, k=8, seed_grad=None):
    p = np.asarray(th).shape[1]
    total = int(off[-1])
    paths = torch.empty((2 + p, total), dtype=torch.float32, device="cuda")
    v, d0, dth = sl.seven_league_adjoint(model, net, _dev(th), _dev(y0), _dev(off, torch.int64), T, n_steps, m,
                                         seed, K, ckpt_k=k, out_paths=paths,
                                         seed_grad=None if seed_grad is None else _dev(seed_grad, torch.float64))
    torch.cuda.synchronize()
    return v.cpu().numpy(), d0.cpu().numpy(), dth.cpu().numpy(), paths.cpu().numpy()


def _check_paths(orc, paths, model, P, th, y0, off, T, n_steps, m, seed, K, d_in, act=0, tol=1e-5):
    yt, val, g = orc.seven_league_payoff_grad(model, P, th, y0, off, T, n_steps, m, seed, K, d_in=d_in, act=act)
    far = np.abs(yt - K) > 1e-4
    assert far.mean() > 0.95
    assert np.allclose(paths[0][far], val[far], rtol=tol, atol=tol)
    for c in range(g.shape[1]):
        a, b = paths[1 + c][far], g[far, c]
        assert np.abs(a - b).max() <= tol * (np.abs(b).max() + 1.0), (c, np.abs(a - b).max())
    return yt, val, g


def test_exact_gbm_paths(sl, orc):
    th = np.array([[0.1, 0.3], [0.05, 0.45]], np.float32)
    y0 = np.array([1.0, 0.9], np.float32)
    off = W.offsets_from_counts([3000, 2011])
    v, d0, dth, paths = _adj(sl, 1, None, th, y0, off, 1.0, 16, 7, 3, 1.0)
    _check_paths(orc, paths, 1, None, th, y0, off, 1.0, 16, 7, 3, 1.0, d_in=4)


def test_exact_ou_paths(sl, orc):
    th = np.array([[0.5, 0.4, 1.3]], np.float32)
    off = W.offsets_from_counts([4001])
    v, d0, dth, paths = _adj(sl, 2, None, th, [1.0], off, 2.0, 12, 5, 5, 0.8)
    _check_paths(orc, paths, 2, None, th, [1.0], off, 2.0, 12, 5, 5, 0.8, d_in=5)


@pytest.mark.parametrize("act", [0, 1])
def test_mlp_paths(sl, orc, act):
    d_in, m = 4, 7
    P = W.xavier_params(d_in, m, seed=5)
    net = sl.make_net(_dev(P), d_in, m, act=act)
    th = W.gbm_online_thetas(3)
    off = W.offsets_from_counts([700, 0, 1333])
    y0 = np.array([0.1, 0.2, 0.05], np.float32)
    K = -1.0 if act == 0 else 0.5
    v, d0, dth, paths = _adj(sl, 0, net, th, y0, off, 2.0, 10, m, 2, K, k=4)
    _check_paths(orc, paths, 0, P.astype(np.float64), th, y0, off, 2.0, 10, m, 2, K, d_in=d_in, act=act)


def test_checkpoint_interval_invariance(sl, orc):
    d_in, m = 5, 7
    P = W.xavier_params(d_in, m, seed=6)
    net = sl.make_net(_dev(P), d_in, m)
    b = W.cir_batched(n_sets=5, lo_exp=2, hi_exp=3)
    ref = None
    for k in (1, 3, 8, 16, 20):
        out = _adj(sl, 0, net, b["theta"], b["Y0"], b["offsets"], 4.0, 20, m, 1, -5.0, k=k)[3]
        if ref is None:
            ref = out
        assert np.array_equal(out, ref), k


def test_set_means_and_seed_grad(sl, orc):
    th = np.array([[0.1, 0.3], [0.02, 0.2], [0.15, 0.5]], np.float32)
    y0 = np.array([1.0, 1.1, 0.9], np.float32)
    off = W.offsets_from_counts([1000, 1, 2500])
    v, d0, dth, paths = _adj(sl, 1, None, th, y0, off, 1.0, 8, 5, 9, 1.0)
    for s in range(3):
        seg = slice(off[s], off[s + 1])
        assert v[s] == pytest.approx(paths[0][seg].astype(np.float64).mean(), rel=1e-12, abs=1e-15)
        assert d0[s] == pytest.approx(paths[1][seg].astype(np.float64).mean(), rel=1e-12, abs=1e-15)
        for c in range(2):
            assert dth[s, c] == pytest.approx(paths[2 + c][seg].astype(np.float64).mean(), rel=1e-12, abs=1e-15)
    sg = np.array([2.0, -1.0, 0.5])
    v2, d02, dth2, _ = _adj(sl, 1, None, th, y0, off, 1.0, 8, 5, 9, 1.0, seed_grad=sg)
    assert np.array_equal(v2, v)
    assert np.allclose(d02, d0 * sg, rtol=1e-15) and np.allclose(dth2, dth * sg[:, None], rtol=1e-15)


def test_vs_central_differences(sl, orc):
    """Path-mean sensitivities vs central differences of the oracle's FP64 mean."""
    d_in, m, n, T, n_steps, K = 4, 7, 20000, 2.0, 8, 1.0
    P = W.xavier_params(d_in, m, seed=0)
    Pd = P.astype(np.float64)
    rng = np.random.default_rng(0)
    # a network whose paths move like a diffusion: y_j = Y * (1 + small net)
    net = sl.make_net(_dev(P), d_in, m)
    th = np.array([[0.1, 0.3]], np.float32)
    off = W.offsets_from_counts([n])
    v, d0, dth, _ = _adj(sl, 0, net, th, [1.0], off, T, n_steps, m, 4, K)

    def mean_payoff(y0, t):
        yt = orc.seven_league_paths(0, Pd, [t], [y0], off, T, n_steps, m, 4, d_in=d_in)
        return np.maximum(yt - K, 0).mean()
    h = 1e-5
    fd0 = (mean_payoff(1.0 + h, th[0]) - mean_payoff(1.0 - h, th[0])) / (2 * h)
    assert d0[0] == pytest.approx(fd0, rel=1e-3, abs=1e-6)
    for c in range(2):
        tp, tm = th[0].astype(np.float64).copy(), th[0].astype(np.float64).copy()
        tp[c] += h
        tm[c] -= h
        fd = (mean_payoff(1.0, tp) - mean_payoff(1.0, tm)) / (2 * h)
        assert dth[0, c] == pytest.approx(fd, rel=1e-3, abs=1e-6), c


def test_black_scholes_gbm_exact(sl, orc):
    mu, sg, T, K, m, n_steps, n = 0.1, 0.3, 1.0, 1.0, 7, 64, 1_000_000
    off = W.offsets_from_counts([n])
    v, d0, dth, paths = _adj(sl, 1, None, [[mu, sg]], [1.0], off, T, n_steps, m, 21, K, k=8)
    d1 = (math.log(1.0 / K) + (mu + 0.5 * sg * sg) * T) / (sg * math.sqrt(T))
    d2 = d1 - sg * math.sqrt(T)
    want = {"price": math.exp(mu * T) * stats.norm.cdf(d1) - K * stats.norm.cdf(d2),
            "delta": math.exp(mu * T) * stats.norm.cdf(d1),
            "dmu": T * math.exp(mu * T) * stats.norm.cdf(d1),
            "vega": math.exp(mu * T) * stats.norm.pdf(d1) * math.sqrt(T)}
    got = {"price": (v[0], paths[0]), "delta": (d0[0], paths[1]), "dmu": (dth[0, 0], paths[2]),
           "vega": (dth[0, 1], paths[3])}
    for key, (est, per_path) in got.items():
        se = per_path.astype(np.float64).std(ddof=1) / math.sqrt(n)
        assert abs(est - want[key]) < 4 * se + 2e-4, (key, est, want[key], se)


def test_cir_adjoint_workload(sl, orc):
    """CIR network (d_in = 5), 64 steps, checkpoint every 8: K = 1 lies far above the
    CIR range (every path out of the money: all sensitivities exactly 0); K = ybar is
    the meaningful case, checked path by path."""
    d_in, m = 5, 7
    P = W.xavier_params(d_in, m, seed=2)
    net = sl.make_net(_dev(P), d_in, m)
    th = np.array([[1.0, 0.1, 0.3]], np.float32)
    off = W.offsets_from_counts([3000])
    v, d0, dth, paths = _adj(sl, 0, net, th, [0.1], off, 1.0, 64, m, 8, 1.0)
    yt = orc.seven_league_paths(0, P.astype(np.float64), th, [0.1], off, 1.0, 64, m, 8, d_in=d_in)
    if yt.max() < 1.0 - 1e-3:
        assert v[0] == 0 and d0[0] == 0 and np.all(dth == 0)
    v, d0, dth, paths = _adj(sl, 0, net, th, [0.1], off, 1.0, 64, m, 8, float(np.median(yt)))
    _check_paths(orc, paths, 0, P.astype(np.float64), th, [0.1], off, 1.0, 64, m, 8, float(np.median(yt)),
                 d_in=d_in)


def test_autograd_function(sl, orc):
    th = _dev([[0.1, 0.3], [0.05, 0.2]]).requires_grad_(True)
    y0 = _dev([1.0, 1.2]).requires_grad_(True)
    off = _dev(W.offsets_from_counts([5000, 3000]), torch.int64)
    kw = dict(model=sl.MODEL_GBM_EXACT, path_offsets=off, T=1.0, n_steps=16, m=7, seed=3, K=1.0)
    val = sl.SevenLeagueCall.apply(y0, th, **kw)
    w = torch.tensor([1.0, -2.0], dtype=torch.float64, device="cuda")
    (val * w).sum().backward()
    _, d0, dth = sl.seven_league_adjoint(sl.MODEL_GBM_EXACT, None, th.detach(), y0.detach(), off, 1.0, 16, 7, 3, 1.0)
    assert torch.allclose(y0.grad.double(), d0 * w, rtol=1e-6)
    assert torch.allclose(th.grad.double(), dth * w[:, None], rtol=1e-6)
