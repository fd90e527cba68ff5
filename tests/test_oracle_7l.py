"""Pins of the oracle's online 7L chain (Algorithm I steps 2-8) and its
pathwise sensitivities.

* Exact-collocation GBM: since m-point Gauss-Hermite quadrature integrates
  polynomials of degree <= 2m-1 exactly and g_m has degree m-1,
  E[Y_{i+1} | Y_i] = Y_i c and E[Y_{i+1}^2 | Y_i] = Y_i^2 d with
  c = sum w_j e^{a + b x_j}, d = sum w_j e^{2a + 2b x_j}; so the chain's
  E[Y_T] = Y0 c^N and E[Y_T^2] = Y0^2 d^N exactly (nodes from numpy).
* Exact-collocation OU (Eq. 6.5/6.6): the collocation points are linear in
  x_j, so g_m reproduces the exact OU transition, and each path equals the
  exact solution (6.6) driven by the same normals, for any step size.
* MLP model: a hand-built ReLU network that computes the exact OU map
  reproduces the OU_EXACT paths (checks feature order Y, dt, theta).
* Batched sets: a set's paths do not depend on the other sets (empty sets
  before it give identical results).
* Sensitivities: dY_T/d(Y0, theta) vs central finite differences of the
  oracle's own path values, and GBM_EXACT call price/delta/vega/rho-in-mu
  vs closed-form (undiscounted) Black-Scholes within Monte Carlo error.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e
from scipy import stats

from paper_2302_05170_b300 import workloads as W


def _gbm_cd(mu, sg, dt, m):
    x, w = hermite_e.hermegauss(m)
    w = w / w.sum()
    a, b = (mu - 0.5 * sg * sg) * dt, sg * math.sqrt(dt)
    return float(np.dot(w, np.exp(a + b * x))), float(np.dot(w, np.exp(2 * a + 2 * b * x)))


@pytest.mark.parametrize("m,n_steps", [(5, 2), (7, 16)])
def test_gbm_exact_chain_moments(orc, m, n_steps):
    mu, sg, Y0, T, n = 0.1, 0.3, 1.0, 1.0, 200_000
    off = [0, n]
    mean, var = orc.seven_league_moments(1, None, [[mu, sg]], [Y0], off, T, n_steps, m, seed=1)
    c, d = _gbm_cd(mu, sg, T / n_steps, m)
    e1, e2 = Y0 * c ** n_steps, Y0 ** 2 * d ** n_steps
    se = math.sqrt((e2 - e1 ** 2) / n)
    assert abs(mean[0] - e1) < 4 * se
    assert var[0] == pytest.approx(e2 - e1 ** 2, rel=0.02)
    # the chain's mean is close to the lognormal one (small polynomial bias)
    assert e1 == pytest.approx(Y0 * math.exp(mu * T), rel=1e-6)


@pytest.mark.parametrize("n_steps", [1, 4, 64])
def test_ou_exact_chain_is_pathwise_exact(orc, n_steps):
    yb, sg, lam, Y0, T, m = 0.5, 0.4, 1.3, 2.0, 3.0, 5
    n = 300
    yt, grid = orc.seven_league_paths(2, None, [[yb, sg, lam]], [Y0], [0, n], T, n_steps, m,
                                      seed=7, grid=True)
    dt = T / n_steps
    e1 = math.exp(-lam * dt)
    s = sg * math.sqrt((1 - math.exp(-2 * lam * dt)) / (2 * lam))
    for q in range(0, n, 37):
        X = orc.normals(7, 0, 0, q, 0, n_steps)
        Y = Y0
        for i in range(n_steps):
            Y = e1 * Y + yb * (1 - e1) + s * X[i]      # Eq. (6.6) over one step
            assert grid[q, i + 1] == pytest.approx(Y, rel=1e-12, abs=1e-12)
        assert yt[q] == pytest.approx(Y, rel=1e-12, abs=1e-12)


def _ou_network(yb, sg, lam, dt, m, shift=50.0):
    """ReLU network (d_in = 2 + 3) whose output equals the exact OU collocation map
    for inputs with Y + shift > 0: unit 0 carries Y + shift through the hidden
    layers (ReLU is the identity there), unit 1 carries theta_0 = Ybar + shift."""
    d_in = 5
    P = np.zeros(W.n_params(d_in, m))
    layers = W.split_params(P, d_in, m)
    (W1, b1) = layers[0]
    W1[0, 0] = 1.0
    b1[0] = shift
    W1[1, 2] = 1.0
    b1[1] = shift
    for (Wl, bl) in layers[1:4]:
        Wl[0, 0] = 1.0
        Wl[1, 1] = 1.0
    (W5, b5) = layers[4]
    x, _ = hermite_e.hermegauss(m)
    e1 = math.exp(-lam * dt)
    s = sg * math.sqrt((1 - math.exp(-2 * lam * dt)) / (2 * lam))
    W5[:, 0] = e1
    W5[:, 1] = 1 - e1
    b5[:] = -shift * e1 - shift * (1 - e1) + s * x
    return P


def test_mlp_model_matches_exact_ou(orc):
    yb, sg, lam, Y0, T, n_steps, m = 0.3, 0.2, 0.8, 1.0, 2.0, 8, 7
    P = _ou_network(yb, sg, lam, T / n_steps, m)
    th = [[yb, 7.0, 9.0]]   # only theta_0 is read by the hand-built network
    n = 200
    a = orc.seven_league_paths(0, P, th, [Y0], [0, n], T, n_steps, m, seed=3, d_in=5)
    b = orc.seven_league_paths(2, None, [[yb, sg, lam]], [Y0], [0, n], T, n_steps, m, seed=3)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-11)


def test_batched_sets_independent(orc):
    P = W.xavier_params(4, 7, seed=0)
    th = np.array([[0.1, 0.2], [0.05, 0.4], [0.15, 0.3]])
    y0 = [1.0, 0.8, 1.2]
    counts = [50, 0, 70]
    off = W.offsets_from_counts(counts)
    full = orc.seven_league_paths(0, P, th, y0, off, 2.0, 4, 7, seed=5, d_in=4)
    # set 2 alone, with empty sets 0 and 1 in front of it
    off2 = W.offsets_from_counts([0, 0, 70])
    alone = orc.seven_league_paths(0, P, th, y0, off2, 2.0, 4, 7, seed=5, d_in=4)
    assert np.array_equal(full[50:], alone)
    # selected indices give the same values as the full evaluation
    idx = np.array([0, 49, 50, 119])
    sel = orc.seven_league_paths(0, P, th, y0, off, 2.0, 4, 7, seed=5, d_in=4, idx=idx)
    assert np.array_equal(sel, full[idx])


def _fd_check(orc, model, P, th, Y0, T, n_steps, m, K, d_in, h=1e-6):
    n = 64
    off = [0, n]
    yt, val, g = orc.seven_league_payoff_grad(model, P, [th], [Y0], off, T, n_steps, m, 11, K,
                                              d_in=d_in)
    def paths(th_, y0_):
        return orc.seven_league_paths(model, P, [th_], [y0_], off, T, n_steps, m, 11, d_in=d_in)
    cols = [(paths(th, Y0 + h) - paths(th, Y0 - h)) / (2 * h)]
    for k in range(len(th)):
        tp, tm = list(th), list(th)
        tp[k] += h
        tm[k] -= h
        cols.append((paths(tp, Y0) - paths(tm, Y0)) / (2 * h))
    fd = np.stack(cols, 1)
    itm = yt > K
    assert np.allclose(g[itm], fd[itm], rtol=2e-5, atol=1e-7)
    assert np.all(g[~itm] == 0)
    assert np.allclose(val, np.maximum(yt - K, 0))


def test_sensitivities_vs_fd_exact_models(orc):
    _fd_check(orc, 1, None, [0.1, 0.3], 1.0, 1.0, 8, 7, K=0.9, d_in=4)
    _fd_check(orc, 2, None, [0.5, 0.4, 1.3], 1.0, 2.0, 6, 5, K=0.7, d_in=5)


def test_sensitivities_vs_fd_mlp(orc):
    P = W.xavier_params(4, 7, seed=0).astype(np.float64)
    # scale the output layer so the paths move: y_j ~ Y + small net output
    _fd_check(orc, 0, P, [0.1, 0.3], 1.0, 2.0, 5, 7, K=-10.0, d_in=4)
    P5 = W.xavier_params(5, 7, seed=1).astype(np.float64)
    _fd_check(orc, 0, P5, [1.0, 0.1, 0.3], 0.1, 1.0, 4, 7, K=-10.0, d_in=5)


def test_black_scholes_gbm_exact(orc):
    mu, sg, Y0, T, K, m, n_steps, n = 0.1, 0.3, 1.0, 1.0, 1.0, 7, 64, 100_000
    yt, val, g = orc.seven_league_payoff_grad(1, None, [[mu, sg]], [Y0], [0, n], T, n_steps, m,
                                              21, K)
    d1 = (math.log(Y0 / K) + (mu + 0.5 * sg * sg) * T) / (sg * math.sqrt(T))
    d2 = d1 - sg * math.sqrt(T)
    price = Y0 * math.exp(mu * T) * stats.norm.cdf(d1) - K * stats.norm.cdf(d2)
    delta = math.exp(mu * T) * stats.norm.cdf(d1)
    vega = Y0 * math.exp(mu * T) * stats.norm.pdf(d1) * math.sqrt(T)
    dmu = T * Y0 * math.exp(mu * T) * stats.norm.cdf(d1)
    for est, want in [(val, price), (g[:, 0], delta), (g[:, 2], vega), (g[:, 1], dmu)]:
        se = est.std(ddof=1) / math.sqrt(n)
        assert abs(est.mean() - want) < 4 * se + 2e-4, (est.mean(), want, se)


def test_relu_margin_pins(orc):
    """ReLU margin (min |hidden pre-activation| along a path):
    (a) all weights 0: every pre-activation is its bias, so the margin is min |b|;
    (b) only layer 1 active (W2..W4 = 0, b2..b4 = 10): the margin is the brute-force
        min over steps i < n_steps and units of |W1 f(Y_i) + b1|, with Y_i from the
        oracle's own path grid (Y_n does not enter: no network call is made there)."""
    d_in, m, w = 4, 5, orc.WIDTH
    n_p = orc.n_params(d_in, m)
    rng = np.random.default_rng(3)
    P = np.zeros(n_p)
    o1 = w * d_in
    bias_idx = [o1 + np.arange(w)]
    o = o1 + w
    for _ in range(3):
        bias_idx.append(o + w * w + np.arange(w))
        o += w * w + w
    for bi in bias_idx:
        P[bi] = rng.uniform(-1, 1, w)
    th = np.array([[0.1, 0.3]])
    off = [0, 20]
    mg = orc.seven_league_relu_margin(P, th, [1.0], off, 1.0, 3, m, 1, d_in=d_in)
    assert np.all(mg == min(np.abs(P[bi]).min() for bi in bias_idx))
    # (b)
    P2 = np.zeros(n_p)
    P2[:o1] = rng.normal(0, 0.5, o1)
    P2[bias_idx[0]] = rng.normal(0, 0.3, w)
    for bi in bias_idx[1:]:
        P2[bi] = 10.0
    P2[o:o + m * w] = rng.normal(0, 0.3, m * w)    # output layer: paths move
    n_steps = 6
    _, grid = orc.seven_league_paths(0, P2, th, [1.0], off, 1.0, n_steps, m, 2, d_in=d_in, grid=True)
    mg = orc.seven_league_relu_margin(P2, th, [1.0], off, 1.0, n_steps, m, 2, d_in=d_in)
    W1, b1 = P2[:o1].reshape(w, d_in), P2[bias_idx[0]]
    for k in range(20):
        f = np.stack([grid[k, :n_steps], np.full(n_steps, 1.0 / n_steps), np.full(n_steps, 0.1),
                      np.full(n_steps, 0.3)], 1)
        z = f @ W1.T + b1
        assert mg[k] == pytest.approx(np.abs(z).min(), rel=1e-12, abs=1e-15)
