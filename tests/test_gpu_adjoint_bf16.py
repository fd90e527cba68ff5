"""GPU parity of the BF16 tensor-core adjoint (network model, ReLU or Softplus)
against the FP64 oracle run on the same BF16-valued weights and biases.

The tensor-core form samples the same paths as the BF16 sampler and
back-propagates through the same BF16 weights with BF16 hi + lo cotangents and
FP32 accumulation.  Its per-path values are checked like the sampler's:

* payoff f(Y_T): |a - b| / (|b| + 1) <= 2e-3, gated on paths whose normals stay
  within |X| <= 4 plus the 99.99th percentile over all paths;
* sensitivities f'(Y_T) dY_T/d(Y0, theta): the ReLU network is piecewise
  linear, so its derivative jumps where a hidden pre-activation changes sign.
  Activations carry 16 significant bits (BF16 hi + lo), so a pre-activation
  moves by about 1e-5 of its scale; on a path whose smallest |pre-activation|
  (the oracle's ReLU margin) exceeds MARGIN = 2e-4 both sides follow the same
  linear pieces and the same 2e-3 gate applies.  Paths with a smaller margin
  may follow a different piece; over all paths (far from the payoff kink) the
  sensitivities must still agree within the gate for at least 97% of paths;
* Softplus networks are smooth: every path away from the payoff kink is held to the
  2e-3 gate (no margin selection);
* per-set means: the kernel's FP64 set means equal the means of its own per-path values
  (rel 1e-12); against the oracle, the means over a set's paths with margin >= MARGIN (away
  from the kink) agree within 2e-3 of (mean |per-path value| + 0.1).  Over all paths the means
  are not compared: a path on another linear piece moves a mean by its own jump (up to several
  times the typical per-path value) over the path count.
"""
import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W
from tests.helpers import flat_sets, gate, max_abs_normals, rel_err, with_biases

pytestmark = pytest.mark.gpu
TOL = 2e-3
MARGIN = 2e-4
MIN_AGREE = 0.97


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _thetas(n_sets, p, seed):
    if p == 2:
        return W.gbm_online_thetas(n_sets)
    return np.random.default_rng(seed).uniform(0.05, 0.4, (n_sets, p)).astype(np.float32)


def _adj(sl, P, d_in, m, th, y0, off, T, n_steps, seed, K, k, prec, act=0):
    net = sl.make_net(_dev(P), d_in, m, act=act, prec=prec)
    p = d_in - 2
    total = int(off[-1])
    paths = torch.empty((2 + p, total), dtype=torch.float32, device="cuda")
    ws = torch.empty(sl.adjoint_workspace_size(total, len(off) - 1, n_steps, k, p), dtype=torch.uint8,
                     device="cuda")
    v, d0, dth = sl.seven_league_adjoint(sl.MODEL_MLP, net, _dev(th), _dev(y0), _dev(off, torch.int64), T,
                                         n_steps, m, seed, K, ckpt_k=k, out_paths=paths, ws=ws)
    torch.cuda.synchronize()
    assert sl.workspace_status(ws) == 0
    return v.cpu().numpy(), d0.cpu().numpy(), dth.cpu().numpy(), paths.cpu().numpy()


def _strike(orc, P, d_in, m, th, y0, off, T, n_steps, seed, idx=None, act=0):
    """A strike near the median of the oracle's Y_T (so about half the paths are in the money)."""
    Pb = W.bf16_round(P).astype(np.float64)
    yt = orc.seven_league_paths(0, Pb, th, y0, off, T, n_steps, m, seed, d_in=d_in, idx=idx, act=act)
    return float(np.median(yt))


def _check(orc, P, d_in, m, th, y0, off, T, n_steps, seed, K, got, act=0):
    v, d0, dth, paths = got
    Pb = W.bf16_round(P).astype(np.float64)
    yt, val, g = orc.seven_league_payoff_grad(0, Pb, th, y0, off, T, n_steps, m, seed, K, d_in=d_in, act=act)
    assert 0.2 < np.mean(val > 0) < 0.8          # a non-trivial mix of in- and out-of-the-money paths
    idx = np.arange(len(yt))
    s, q = flat_sets(off, idx)
    mx = max_abs_normals(orc, seed, 0, s, q, n_steps)
    ok, *info = gate(rel_err(paths[0], val, 1.0), mx, TOL)
    assert ok, ("payoff", info)
    far = np.abs(yt - K) > 5 * TOL * (np.abs(yt) + 1.0)
    if act == 0:
        mg = orc.seven_league_relu_margin(Pb, th, y0, off, T, n_steps, m, seed, d_in=d_in)
        sure = far & (mg >= MARGIN)
    else:                                       # smooth network: no linear pieces to switch
        sure = far
    for c in range(g.shape[1]):
        err = rel_err(paths[1 + c], g[:, c], 1.0)
        if sure.any():
            ok, *info = gate(err[sure], mx[sure], TOL)
            assert ok, ("sensitivity", c, "margin >= %g" % MARGIN, int(sure.sum()), info)
        agree = np.mean(err[far] <= TOL)
        assert agree >= MIN_AGREE, ("sensitivity", c, agree)
    for st in range(len(off) - 1):
        seg = slice(off[st], off[st + 1])
        if off[st + 1] == off[st]:
            assert v[st] == 0 and d0[st] == 0 and np.all(dth[st] == 0)
            continue
        # the kernel's set means are the FP64 means of its own per-path values
        assert v[st] == pytest.approx(paths[0][seg].astype(np.float64).mean(), rel=1e-12, abs=1e-15)
        assert d0[st] == pytest.approx(paths[1][seg].astype(np.float64).mean(), rel=1e-12, abs=1e-15)
        for c in range(dth.shape[1]):
            assert dth[st, c] == pytest.approx(paths[2 + c][seg].astype(np.float64).mean(), rel=1e-12, abs=1e-15)
        # against the oracle: means over the set's paths away from ReLU switches and the kink
        sel = sure[seg]
        if sel.sum() < 10:
            continue
        for c in range(g.shape[1]):
            a, b = paths[1 + c][seg][sel].astype(np.float64), g[seg, c][sel]
            assert abs(a.mean() - b.mean()) <= TOL * (np.abs(b).mean() + 0.1), (st, c)
    return sure.mean()


@pytest.mark.parametrize("d_in,m,counts,n_steps,k", [
    (4, 7, [3000, 129, 5000], 16, 4),
    (5, 5, [0, 1, 4000, 383], 10, 3),
    (7, 8, [2000, 0], 6, 8),
    (3, 2, [1500], 6, 32),
    (4, 7, [37], 1, 1),
])
def test_paths_vs_oracle(sl, orc, d_in, m, counts, n_steps, k):
    P = W.xavier_params(d_in, m, seed=d_in + m)
    th = _thetas(len(counts), d_in - 2, m)
    off = W.offsets_from_counts(counts)
    y0 = np.linspace(0.9, 1.1, len(counts)).astype(np.float32)
    K = _strike(orc, P, d_in, m, th, y0, off, 2.0, n_steps, 5)
    got = _adj(sl, P, d_in, m, th, y0, off, 2.0, n_steps, 5, K, k, sl.PREC_BF16)
    _check(orc, P, d_in, m, th, y0, off, 2.0, n_steps, 5, K, got)


@pytest.mark.parametrize("d_in,m,counts,n_steps,k", [
    (4, 7, [3000, 129, 5000], 16, 4),
    (5, 5, [0, 1, 4000, 383], 10, 3),
    (3, 2, [1500], 6, 32),
    (4, 7, [37], 1, 1),
    (6, 8, [2500], 9, 9),
])
def test_softplus_paths_vs_oracle(sl, orc, d_in, m, counts, n_steps, k):
    """Softplus network (the paper's activation): the reverse sweep recomputes each layer's
    pre-activation; per-path sensitivities on every path away from the payoff kink."""
    P = W.xavier_params(d_in, m, seed=20 + d_in + m)
    th = _thetas(len(counts), d_in - 2, m)
    off = W.offsets_from_counts(counts)
    y0 = np.linspace(0.9, 1.1, len(counts)).astype(np.float32)
    K = _strike(orc, P, d_in, m, th, y0, off, 2.0, n_steps, 5, act=1)
    got = _adj(sl, P, d_in, m, th, y0, off, 2.0, n_steps, 5, K, k, sl.PREC_BF16, act=1)
    assert _check(orc, P, d_in, m, th, y0, off, 2.0, n_steps, 5, K, got, act=1) > 0.9


@pytest.mark.parametrize("act", [0, 1])
@pytest.mark.parametrize("d_in,m,counts,n_steps,k", [
    (4, 7, [3000, 129, 2500], 12, 4),
    (7, 5, [2000, 700], 6, 3),
])
def test_biases_paths_vs_oracle(sl, orc, act, d_in, m, counts, n_steps, k):
    """Nonzero biases (up to 1.5 in magnitude) in every layer, both activations: the forward
    sweep and the reverse sweep's recomputes carry them on the bias units (the Softplus form's in
    base 2, log2(e) as a BF16 hi + lo pair), the backward chain meets them as zero rows."""
    P = with_biases(W.xavier_params(d_in, m, seed=50 + d_in + m), W.layer_shapes(d_in, m), 1.5, seed=d_in * m)
    th = _thetas(len(counts), d_in - 2, m)
    off = W.offsets_from_counts(counts)
    y0 = np.linspace(0.9, 1.1, len(counts)).astype(np.float32)
    K = _strike(orc, P, d_in, m, th, y0, off, 2.0, n_steps, 5, act=act)
    got = _adj(sl, P, d_in, m, th, y0, off, 2.0, n_steps, 5, K, k, sl.PREC_BF16, act=act)
    sure = _check(orc, P, d_in, m, th, y0, off, 2.0, n_steps, 5, K, got, act=act)
    if act == 1:
        assert sure > 0.9


def test_softplus_bf16_vs_fp32_forms(sl, orc):
    """Both forms of a Softplus network on the same paths: the set sensitivities agree to the
    BF16 weight quantisation (each form against the oracle on its own weights above)."""
    P = W.xavier_params(4, 7, seed=31)
    th = _thetas(2, 2, 7)
    off = W.offsets_from_counts([20000, 15000])
    y0 = np.array([1.0, 0.95], np.float32)
    K = _strike(orc, P, 4, 7, th, y0, off, 2.0, 16, 6, idx=np.arange(0, 35000, 7), act=1)
    a = _adj(sl, P, 4, 7, th, y0, off, 2.0, 16, 6, K, 8, sl.PREC_BF16, act=1)
    b = _adj(sl, P, 4, 7, th, y0, off, 2.0, 16, 6, K, 8, sl.PREC_FP32, act=1)
    for x, y in zip(a[:3], b[:3]):
        assert np.allclose(x, y, rtol=0.05, atol=0.02 * np.abs(y).max() + 1e-6), (x, y)


def _ou_network(yb, sg, lam, dt, m, shift=2.0, noise=0.0, seed=0):
    """ReLU network (d_in = 5) whose output is the exact OU collocation map for
    Y + shift > 0: unit 0 carries Y + shift, unit 1 carries theta_0 + shift through
    the hidden layers; every other unit has bias -1 (off, far from its switch).
    With noise > 0 every weight gets N(0, noise^2) added (a diffusion-like network
    whose other units switch along the paths)."""
    from numpy.polynomial import hermite_e
    d_in = 5
    P = np.zeros(W.n_params(d_in, m))
    layers = W.split_params(P, d_in, m)
    for li, (Wl, bl) in enumerate(layers[:4]):
        bl[:] = -1.0
        bl[0] = bl[1] = shift if li == 0 else 0.0
        if li == 0:
            Wl[0, 0] = Wl[1, 2] = 1.0
        else:
            Wl[0, 0] = Wl[1, 1] = 1.0
    W5, b5 = layers[4]
    x, _ = hermite_e.hermegauss(m)
    e1 = np.exp(-lam * dt)
    s = sg * np.sqrt((1 - np.exp(-2 * lam * dt)) / (2 * lam))
    W5[:, 0] = e1
    W5[:, 1] = 1 - e1
    b5[:] = -shift + s * x
    if noise:
        P += np.random.default_rng(seed).normal(0.0, noise, P.shape)
    return P.astype(np.float32)


@pytest.mark.parametrize("noise", [0.0, 0.01])
def test_ou_network(sl, orc, noise):
    """A network that moves paths like an OU diffusion: dY_T/dY0 = e^{-lambda T}-like
    products and d/dYbar through a second unit.  Without noise every mask is fixed
    (margins >= 1), so all far-from-kink paths fall under the strict gate."""
    yb, sg, lam, T, n_steps, m = 0.3, 0.2, 0.8, 2.0, 8, 7
    P = _ou_network(yb, sg, lam, T / n_steps, m, noise=noise)
    th = np.array([[yb, sg, lam], [0.5, sg, lam]], np.float32)
    off = W.offsets_from_counts([3000, 2000])
    y0 = np.array([1.0, 0.4], np.float32)
    K = _strike(orc, P, 5, m, th, y0, off, T, n_steps, 4)
    got = _adj(sl, P, 5, m, th, y0, off, T, n_steps, 4, K, 3, sl.PREC_BF16)
    sure = _check(orc, P, 5, m, th, y0, off, T, n_steps, 4, K, got)
    if noise == 0.0:
        assert sure > 0.9
        assert np.all(np.abs(got[2][:, 1:]) < 1e-6)   # sigma, lambda do not enter this network


def test_trained_network(sl, orc):
    """A network trained on GBM labels (the online workload's kind of weights)."""
    from paper_2302_05170_b300 import pipeline
    P = pipeline.train_gbm_online_network(n_rows=1 << 12, n_steps=3000)[0].cpu().numpy()
    th = W.gbm_online_thetas(4)
    off = W.offsets_from_counts([4000, 3000, 2000, 1000])
    y0 = np.ones(4, np.float32)
    K = _strike(orc, P, 4, 7, th, y0, off, 2.0, 16, 11)
    got = _adj(sl, P, 4, 7, th, y0, off, 2.0, 16, 11, K, 8, sl.PREC_BF16)
    _check(orc, P, 4, 7, th, y0, off, 2.0, 16, 11, K, got)


def test_checkpoint_interval_invariance(sl, orc):
    """The recomputed segments replay the forward sweep's arithmetic: every k gives the
    same per-path values (to FP32 rounding: the sweeps are separate code sites)."""
    P = W.xavier_params(5, 7, seed=6)
    b = W.cir_batched(n_sets=5, lo_exp=2, hi_exp=3)
    ref = None
    K = _strike(orc, P, 5, 7, b["theta"], b["Y0"], b["offsets"], 4.0, 20, 1)
    for k in (1, 3, 8, 20, 32):
        out = _adj(sl, P, 5, 7, b["theta"], b["Y0"], b["offsets"], 4.0, 20, 1, K, k, sl.PREC_BF16)[3]
        if ref is None:
            ref = out
            assert 0.2 < np.mean(ref[0] > 0) < 0.8
        assert np.all(np.abs(out - ref) <= 1e-6 * (np.abs(ref) + 1.0)), k


def test_payoff_matches_sampler(sl, orc):
    """The adjoint's forward sweep is the BF16 sampler's: f(Y_T) = max(Y_T - K, 0) of
    seven_league_simulate_batched's Y_T on the same inputs."""
    P = W.xavier_params(4, 7, seed=3)
    th = W.gbm_online_thetas(3)
    off = W.offsets_from_counts([5000, 777, 12000])
    y0 = np.ones(3, np.float32)
    K = _strike(orc, P, 4, 7, th, y0, off, 2.0, 16, 9, idx=np.arange(0, int(off[-1]), 17))
    paths = _adj(sl, P, 4, 7, th, y0, off, 2.0, 16, 9, K, 8, sl.PREC_BF16)[3]
    net = sl.make_net(_dev(P), 4, 7, prec=sl.PREC_BF16)
    yt = torch.empty(int(off[-1]), dtype=torch.float32, device="cuda")
    sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(th), _dev(y0), _dev(off, torch.int64), 2.0, 16, 7,
                                     9, out_YT=yt)
    f = np.maximum(yt.cpu().numpy() - K, 0.0)
    assert 0.2 < np.mean(f > 0) < 0.8
    assert np.all(np.abs(paths[0] - f) <= 1e-6 * (np.abs(f) + 1.0))


def test_bf16_vs_fp32_forms(sl, orc):
    """Both network forms on the same BF16-valued weights: per-set means agree to the
    BF16 tolerance."""
    P = W.bf16_round(W.xavier_params(4, 7, seed=4)).astype(np.float32)
    th = W.gbm_online_thetas(4)
    off = W.offsets_from_counts([20000] * 4)
    y0 = np.ones(4, np.float32)
    K = _strike(orc, P, 4, 7, th, y0, off, 2.0, 16, 2, idx=np.arange(0, int(off[-1]), 37))
    a = _adj(sl, P, 4, 7, th, y0, off, 2.0, 16, 2, K, 8, sl.PREC_BF16)
    b = _adj(sl, P, 4, 7, th, y0, off, 2.0, 16, 2, K, 8, sl.PREC_FP32)
    assert 0.2 < np.mean(a[3][0] > 0) < 0.8
    for x, y in zip(a[:3], b[:3]):
        assert np.all(np.abs(x - y) <= TOL * (np.abs(y) + 0.1))


def test_all_out_of_the_money(sl, orc):
    """K far above every Y_T: all sensitivities are exactly 0 (the reverse sweep is skipped)."""
    P = W.xavier_params(4, 7, seed=5)
    th = W.gbm_online_thetas(2)
    off = W.offsets_from_counts([1000, 300])
    v, d0, dth, paths = _adj(sl, P, 4, 7, th, np.ones(2, np.float32), off, 1.0, 8, 3, 1e6, 8, sl.PREC_BF16)
    assert np.all(v == 0) and np.all(d0 == 0) and np.all(dth == 0) and np.all(paths == 0)


def test_full_size_sampled(sl, orc):
    """1e6 paths x 64 steps, checkpoint every 8 (the bench's adjoint workload), sampled paths."""
    P = W.xavier_params(4, 7, seed=0)
    th = np.array([[0.1, 0.3]], np.float32)
    n = 10 ** 6
    off = W.offsets_from_counts([n])
    rng = np.random.default_rng(2)
    idx = np.unique(np.concatenate([rng.integers(0, n, 2000), [0, n - 1]]))
    K = _strike(orc, P, 4, 7, th, [1.0], off, 1.0, 64, 1, idx=idx)
    v, d0, dth, paths = _adj(sl, P, 4, 7, th, [1.0], off, 1.0, 64, 1, K, 8, sl.PREC_BF16)
    Pb = W.bf16_round(P).astype(np.float64)
    yt, val, g = orc.seven_league_payoff_grad(0, Pb, th, [1.0], off, 1.0, 64, 7, 1, K, idx=idx, d_in=4)
    mx = max_abs_normals(orc, 1, 0, np.zeros(len(idx), int), idx, 64)
    ok, *info = gate(rel_err(paths[0][idx], val, 1.0), mx, TOL)
    assert ok, info
    far = np.abs(yt - K) > 5 * TOL * (np.abs(yt) + 1.0)
    for c in range(3):
        assert np.mean(rel_err(paths[1 + c][idx], g[:, c], 1.0)[far] <= TOL) >= MIN_AGREE, c
    assert np.all(np.isfinite(paths))


@pytest.mark.parametrize("act,seed", [(1, 0), (1, 5), (0, 0), (0, 5), (0, 9)])
def test_set_means_vs_central_differences(sl, orc, act, seed):
    """The tensor-core adjoint's set means (FP64) against central differences of the oracle's FP64
    mean payoff on the same BF16-valued weights and the same normals, h = 1e-5: within 1e-3 relative.
    Softplus networks are smooth; for ReLU networks a path whose pre-activation sits within the BF16
    activations' rounding (~1e-5 of its scale) of zero may follow the neighbouring linear piece, which
    moves a mean by that path's jump over the path count -- within the same 1e-3 here."""
    d_in, m, n, T, n_steps = 4, 7, 20000, 2.0, 8
    P = W.near_affine_params(d_in, m, eps=0.05, seed=seed)      # paths that move like a diffusion
    Pb = W.bf16_round(P).astype(np.float64)
    th = np.array([[0.1, 0.3]], np.float32)
    off = W.offsets_from_counts([n])
    K = _strike(orc, Pb, d_in, m, th, [1.0], off, T, n_steps, 4, act=act)
    v, d0, dth, _ = _adj(sl, P, d_in, m, th, [1.0], off, T, n_steps, 4, K, 8, sl.PREC_BF16, act=act)

    def mean_payoff(y0, t):
        yt = orc.seven_league_paths(0, Pb, [t], [y0], off, T, n_steps, m, 4, d_in=d_in, act=act)
        return np.maximum(yt - K, 0).mean()
    h = 1e-5
    fd = [(mean_payoff(1.0 + h, th[0].astype(np.float64)) - mean_payoff(1.0 - h, th[0].astype(np.float64))) / (2 * h)]
    for c in range(2):
        tp, tm = th[0].astype(np.float64).copy(), th[0].astype(np.float64).copy()
        tp[c] += h
        tm[c] -= h
        fd.append((mean_payoff(1.0, tp) - mean_payoff(1.0, tm)) / (2 * h))
    got = [d0[0], dth[0, 0], dth[0, 1]]
    rel = [abs(g - f) / max(abs(f), 1e-3) for g, f in zip(got, fd)]
    print("adjoint set means", got, "central differences", fd, "relative gaps", rel)
    assert min(abs(f) for f in fd) > 1e-3                       # every sensitivity is a real one
    for g, f in zip(got, fd):
        assert g == pytest.approx(f, rel=1e-3, abs=1e-6)
