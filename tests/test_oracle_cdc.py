"""Pins of the oracle's 7L-CDC chain (the variant discussed with Table 6.1: the per-path
network of Algorithm I step 3 replaced by an interpolation in Y through the marginal
collocation points).

* The interpolation in Y reproduces every polynomial of degree <= m-1 inside the nodes' hull
  (values checked with numpy's polyval), returns row k at Y = z_k, returns row 0 when all
  nodes coincide; beyond the outermost nodes it is a straight line in Y (zero second
  differences) that meets the interpolant at the outermost node and has the slope of the two
  outermost nodes; maps affine in Y are reproduced everywhere, nodes in any order.
* Marginal nodes of the exact models are the exact quantiles of Y_{t_i} at levels Phi(x_k):
  scipy's lognormal (GBM) and normal (OU, Eq. 6.6) quantile functions at numpy's
  Gauss-Hermite nodes; the conditional points at the nodes are the exact conditional
  quantiles from the same scipy functions; step 0 is the point mass at Y0.
* The exact GBM and OU conditional maps are linear in Y, so the interpolation in Y is exact
  and the 7L-CDC chain equals the (separately pinned) 7L chain path by path.
* A ReLU network whose units are all active computes an affine map of its inputs, so its
  7L-CDC chain equals its 7L chain; a network with inactive units does not (the check above
  is not vacuous).  With one step the two chains coincide for any network.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e
from scipy import stats

from paper_2302_05170_b300 import workloads as W


@pytest.mark.parametrize("m", [2, 3, 5, 7, 8])
def test_interpolation_in_y_reproduces_polynomials(orc, m):
    rng = np.random.default_rng(m)
    z = np.sort(rng.uniform(-2.0, 3.0, m))
    coef = rng.normal(size=(m, m))                 # point j is the polynomial coef[j] (degree m-1)
    C = np.array([[np.polyval(coef[j], zk) for j in range(m)] for zk in z])
    for Y in np.concatenate([rng.uniform(z[0], z[-1], 20), z]):
        got = orc.cdc_conditional_points(z, C, Y)
        want = np.array([np.polyval(coef[j], Y) for j in range(m)])
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * np.abs(want).max()), Y
    for k in range(m):
        assert np.array_equal(orc.cdc_conditional_points(z, C, z[k]), C[k])
    assert np.array_equal(orc.cdc_conditional_points(np.full(m, 0.7), C, 5.0), C[0])


@pytest.mark.parametrize("m", [2, 5, 8])
def test_continuation_beyond_the_nodes(orc, m):
    rng = np.random.default_rng(10 + m)
    z = rng.permutation(np.sort(rng.uniform(-1.0, 2.0, m)))          # nodes in no particular order
    coef = rng.normal(size=(m, 3))                                    # quadratic points
    C = np.array([[np.polyval(coef[j], zk) for j in range(m)] for zk in z])
    zs = np.sort(z)
    for edge, inner, side in ((zs[0], zs[1], -1.0), (zs[-1], zs[-2], 1.0)):
        Ys = edge + side * np.array([1e-9, 0.5, 1.0, 1.5, 40.0])
        v = np.array([orc.cdc_conditional_points(z, C, Y) for Y in Ys])
        at_edge = orc.cdc_conditional_points(z, C, edge)
        assert np.allclose(v[0], at_edge, atol=1e-7)                    # continuous at the node
        assert np.allclose(v[1] - 2 * v[2] + v[3], 0.0, atol=1e-9)      # straight line
        slope = (at_edge - orc.cdc_conditional_points(z, C, inner)) / (edge - inner)
        assert np.allclose((v[4] - at_edge) / (Ys[4] - edge), slope, rtol=1e-9)
    lin = rng.normal(size=(m, 2))                                     # affine points: exact everywhere
    CL = np.array([[lin[j, 0] + lin[j, 1] * zk for j in range(m)] for zk in z])
    for Y in (-50.0, -1.3, 0.4, 2.7, 60.0):
        assert np.allclose(orc.cdc_conditional_points(z, CL, Y), lin[:, 0] + lin[:, 1] * Y, rtol=1e-12, atol=1e-12)


def test_interpolation_in_y_is_not_exact_beyond_degree(orc):
    m = 4
    z = np.array([-1.0, 0.0, 0.5, 2.0])
    C = np.stack([z ** m] * m, 1)                  # every point is Y^4, degree m
    assert abs(orc.cdc_conditional_points(z, C, 1.0)[0] - 1.0) > 1e-3


def _nodes(m):
    return hermite_e.hermegauss(m)[0]


def test_exact_gbm_tables(orc):
    m, n_steps, T = 7, 8, 2.0
    th = np.array([[0.1, 0.3], [0.05, 0.45]])
    Y0 = np.array([1.0, 2.5])
    z, C = orc.cdc_tables(orc.MODEL_GBM_EXACT, None, th, Y0, T, n_steps, m)
    x, dt = _nodes(m), T / n_steps
    lev = stats.norm.cdf(x)
    for s, (mu, sg) in enumerate(th):
        assert np.all(z[s, 0] == Y0[s])
        for i in range(n_steps):
            t = i * dt
            if i:
                want = stats.lognorm.ppf(lev, s=sg * math.sqrt(t), scale=Y0[s] * math.exp((mu - sg * sg / 2) * t))
                assert np.allclose(z[s, i], want, rtol=1e-10), (s, i)
            for k in range(m):
                want = stats.lognorm.ppf(lev, s=sg * math.sqrt(dt), scale=z[s, i, k] * math.exp((mu - sg * sg / 2) * dt))
                assert np.allclose(C[s, i, k], want, rtol=1e-10), (s, i, k)


def test_exact_ou_tables(orc):
    m, n_steps, T = 5, 4, 2.0
    th = np.array([[0.5, 0.3, 1.0], [-0.2, 0.15, 1.7]])
    Y0 = np.array([1.5, 0.1])
    z, C = orc.cdc_tables(orc.MODEL_OU_EXACT, None, th, Y0, T, n_steps, m)
    x, dt = _nodes(m), T / n_steps
    lev = stats.norm.cdf(x)

    def ou_q(y, yb, sg, lam, t):
        return stats.norm.ppf(lev, loc=math.exp(-lam * t) * y + yb * (1 - math.exp(-lam * t)),
                              scale=sg * math.sqrt((1 - math.exp(-2 * lam * t)) / (2 * lam)))

    for s, (yb, sg, lam) in enumerate(th):
        for i in range(1, n_steps):
            assert np.allclose(z[s, i], ou_q(Y0[s], yb, sg, lam, i * dt), rtol=1e-10, atol=1e-12)
            for k in range(m):
                assert np.allclose(C[s, i, k], ou_q(z[s, i, k], yb, sg, lam, dt), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("model,theta,Y0,m", [
    (1, [[0.1, 0.3], [0.15, 0.5], [0.0, 0.1]], [1.0, 0.7, 3.0], 7),
    (1, [[0.1, 0.3]], [1.0], 2),
    (2, [[0.5, 0.3, 1.0], [1.0, 0.45, 0.6]], [1.5, -0.5], 5),
    (2, [[0.5, 0.3, 1.0]], [1.5], 8),
])
def test_exact_cdc_chain_equals_7l_chain(orc, model, theta, Y0, m):
    n_sets = len(Y0)
    off = W.offsets_from_counts([700 + 300 * s for s in range(n_sets)])
    for n_steps in (1, 4, 16):
        cdc = orc.cdc_paths(model, None, theta, Y0, off, 2.0, n_steps, m, 11)
        ref = orc.seven_league_paths(model, None, theta, Y0, off, 2.0, n_steps, m, 11)
        assert np.allclose(cdc, ref, rtol=1e-11, atol=1e-11), n_steps


def _affine_net(d_in, m, seed):
    """First-layer bias 10 (|W1| <= 0.34, so every first-layer unit is active while the
    features stay below 20 in magnitude), then positive weights and biases: every ReLU unit
    is active and the network is an affine map of its features."""
    P = W.xavier_params(d_in, m, seed=seed).astype(np.float64)
    out = []
    layers = W.layer_shapes(d_in, m)
    k = 0
    for li, (fo, fi) in enumerate(layers):
        Wl = P[k:k + fo * fi]
        b = np.full(fo, 10.0 if li == 0 else 0.01)
        if li < len(layers) - 1:
            Wl = np.abs(Wl) / fi
        out += [Wl, b]
        k += fo * fi + fo
    return np.concatenate(out)


def test_affine_network_cdc_equals_7l(orc):
    d_in, m = 4, 7
    P = _affine_net(d_in, m, 3)
    th = np.array([[0.1, 0.3], [0.05, 0.2]])
    Y0 = np.array([1.0, 2.0])
    off = W.offsets_from_counts([500, 400])
    assert np.abs(W.split_params(P, d_in, m)[0][0]).max() < 0.34
    cdc, gc = orc.cdc_paths(0, P, th, Y0, off, 2.0, 8, m, 5, d_in=d_in, grid=True)
    ref, gr = orc.seven_league_paths(0, P, th, Y0, off, 2.0, 8, m, 5, d_in=d_in, grid=True)
    z, _ = orc.cdc_tables(0, P, th, Y0, 2.0, 8, m, d_in=d_in)
    assert max(np.abs(gc).max(), np.abs(gr).max(), np.abs(z).max()) < 19.0   # features inside the active box
    assert np.allclose(cdc, ref, rtol=1e-10, atol=1e-10)


def test_nonlinear_network_cdc_differs_but_first_step_agrees(orc):
    d_in, m = 4, 7
    P = W.xavier_params(d_in, m, seed=4)
    th = np.array([[0.1, 0.3]])
    off = W.offsets_from_counts([300])
    one_c = orc.cdc_paths(0, P, th, [1.0], off, 0.5, 1, m, 5, d_in=d_in)
    one_r = orc.seven_league_paths(0, P, th, [1.0], off, 0.5, 1, m, 5, d_in=d_in)
    assert np.array_equal(one_c, one_r)
    cdc = orc.cdc_paths(0, P, th, [1.0], off, 2.0, 8, m, 5, d_in=d_in)
    ref = orc.seven_league_paths(0, P, th, [1.0], off, 2.0, 8, m, 5, d_in=d_in)
    assert np.abs(cdc - ref).max() > 1e-6


def test_marginal_network_argument(orc):
    """The marginal nodes come from the marginal network when one is given."""
    d_in, m = 4, 5
    P, Pm = W.xavier_params(d_in, m, seed=5), W.xavier_params(d_in, m, seed=6)
    th = np.array([[0.1, 0.3]])
    z_same, C_same = orc.cdc_tables(0, P, th, [1.0], 2.0, 4, m, d_in=d_in)
    z_m, C_m = orc.cdc_tables(0, P, th, [1.0], 2.0, 4, m, Pm=Pm, d_in=d_in)
    f = np.array([[1.0, 0.5 * i, 0.1, 0.3] for i in range(1, 4)])
    assert np.allclose(z_m[0, 1:], orc.mlp_forward(Pm, f, d_in, m), rtol=1e-13)
    assert np.allclose(z_same[0, 1:], orc.mlp_forward(P, f, d_in, m), rtol=1e-13)
    assert np.array_equal(C_m[0, 0], C_same[0, 0])


def test_grid_output(orc):
    off = W.offsets_from_counts([50, 30])
    yt, g = orc.cdc_paths(1, None, [[0.1, 0.3], [0.2, 0.2]], [1.0, 2.0], off, 1.0, 6, 5, 3, grid=True)
    assert np.array_equal(g[:, -1], yt)
    assert np.all(g[:50, 0] == 1.0) and np.all(g[50:, 0] == 2.0)
