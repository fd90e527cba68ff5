"""Pins of the oracle's quantile-coordinate 7L-CDC chain (the marginal collocation map
G_i(xi) = sum_k z_k L_k(xi) through the Gauss-Hermite points carries each path as xi; the
conditional points are moved into the next step's coordinate by G_{i+1}^{-1}).

* G interpolates (x_k, z_k) and continues linearly beyond the outer points; where G increases
  (a quantile map) G^{-1} inverts it (G^{-1}(z_k) = x_k, G(G^{-1}(y)) = y inside and outside the
  range); a constant G inverts to 0 and a G that does not increase from its first to its last
  point to NaN.
* The bivariate interpolant reproduces every tensor-product polynomial of degree <= m-1 in each
  variable (numpy polyval), at and away from the nodes, for xi inside [x_0, x_{m-1}]; beyond, it
  is the line in xi through the two outermost node rows.
* The exact OU map makes G linear and the conditional points affine, so the chain equals the
  (separately pinned) 7L chain path by path; sigma = 0 gives the deterministic growth
  Y0 e^{mu T}; the exact GBM chain stays within the interpolation error of the lognormal
  marginal of the 7L GBM chain.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e

from paper_2302_05170_b300 import workloads as W


@pytest.mark.parametrize("m", [2, 5, 7, 8])
def test_G_and_inverse(orc, m):
    x = hermite_e.hermegauss(m)[0]
    z = 0.5 + 0.8 * x + 0.02 * x ** 3              # a quantile-like map: G increases everywhere
    for k in range(m):
        assert orc.cdcq_G(z, x[k]) == pytest.approx(z[k], abs=1e-12)
        assert orc.cdcq_Ginv(z, z[k]) == pytest.approx(x[k], abs=1e-9)
    lo, hi = z[0] - 2.0, z[-1] + 2.0
    for y in np.linspace(lo, hi, 41):
        xi = orc.cdcq_Ginv(z, y)
        assert orc.cdcq_G(z, xi) == pytest.approx(y, abs=1e-9)
    # beyond the range: the lines through the two outermost points
    assert orc.cdcq_Ginv(z, lo) == pytest.approx(x[0] + (lo - z[0]) * (x[1] - x[0]) / (z[1] - z[0]), rel=1e-12)
    assert math.isnan(orc.cdcq_Ginv(z[::-1].copy(), 0.5))
    assert orc.cdcq_Ginv(np.full(m, 0.7), 3.0) == 0.0


@pytest.mark.parametrize("m", [2, 4, 7])
def test_bivariate_interpolation_reproduces_polynomials(orc, m):
    x = hermite_e.hermegauss(m)[0]
    rng = np.random.default_rng(10 + m)
    c = rng.normal(size=(m, m))                      # p(xi, X) = sum_ab c[a, b] xi^a X^b
    p = lambda u, v: sum(c[a, b] * u ** a * v ** b for a in range(m) for b in range(m))
    eta = np.array([[p(x[k], x[j]) for j in range(m)] for k in range(m)])
    for u, v in [(x[0], x[-1]), (0.3 * x[-1], -1.7), (0.8 * x[0], 0.9), (x[-1], 3.3), (0.1, -4.4)]:
        assert orc.cdcq_F(eta, u, v) == pytest.approx(p(u, v), rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("m", [2, 5, 7])
def test_continuation_beyond_the_hull_in_xi(orc, m):
    """Beyond [x_0, x_{m-1}] the interpolant follows the line in xi through the two outermost
    node rows: continuous at the edge, zero second differences, the outer rows' slope."""
    x = hermite_e.hermegauss(m)[0]
    rng = np.random.default_rng(20 + m)
    eta = rng.normal(size=(m, m))
    for X in (-1.3, 0.4, 2.9):
        for edge, inner, side in ((x[0], x[1], -1.0), (x[-1], x[-2], 1.0)):
            us = edge + side * np.array([1e-9, 0.5, 1.0, 1.5])
            v = np.array([orc.cdcq_F(eta, u, X) for u in us])
            at = orc.cdcq_F(eta, edge, X)
            assert v[0] == pytest.approx(at, abs=1e-7)
            assert v[1] - 2 * v[2] + v[3] == pytest.approx(0.0, abs=1e-9)
            slope = (at - orc.cdcq_F(eta, inner, X)) / (edge - inner)
            assert (v[3] - at) / (us[3] - edge) == pytest.approx(slope, rel=1e-9)


@pytest.mark.parametrize("m", [2, 5, 7])
def test_ou_chain_equals_7l_chain(orc, m):
    th, y0 = [[0.5, 0.3, 1.0], [1.0, 0.45, 0.6], [-0.2, 0.2, 1.7]], [1.5, -0.5, 0.0]
    off = W.offsets_from_counts([900, 700, 500])
    for n_steps in (1, 4, 16):
        a = orc.cdcq_paths(2, None, th, y0, off, 2.0, n_steps, m, 11)
        b = orc.seven_league_paths(2, None, th, y0, off, 2.0, n_steps, m, 11)
        assert np.allclose(a, b, rtol=1e-11, atol=1e-11), n_steps


def test_degenerate_and_grid(orc):
    off = W.offsets_from_counts([300, 200])
    yt, g = orc.cdcq_paths(1, None, [[0.1, 0.0], [0.2, 0.0]], [1.0, 2.0], off, 2.0, 8, 7, 3, grid=True)
    assert np.allclose(yt[:300], math.exp(0.2), rtol=1e-12) and np.allclose(yt[300:], 2 * math.exp(0.4), rtol=1e-12)
    assert np.array_equal(g[:, -1], yt) and np.all(g[:300, 0] == 1.0)


def test_gbm_chain_close_to_7l_chain(orc):
    """sigma sqrt(T) up to 0.5: G interpolates the lognormal marginal at 7 points; the paths
    agree with the 7L chain to its interpolation error (mean 1e-3, 99th percentile 1e-2)."""
    th, y0 = [[0.1, 0.3], [0.15, 0.35]], [1.0, 0.7]
    off = W.offsets_from_counts([4000, 3000])
    a = orc.cdcq_paths(1, None, th, y0, off, 2.0, 16, 7, 5)
    b = orc.seven_league_paths(1, None, th, y0, off, 2.0, 16, 7, 5)
    d = np.abs(a - b) / (np.abs(b) + 1.0)
    assert d.mean() < 1e-3 and np.percentile(d, 99) < 1e-2


def test_tables(orc):
    """zn: the exact marginal nodes of t_{i+1}; eta: G_{i+1}^{-1} of the conditional points."""
    th, y0 = [[0.5, 0.3, 1.0]], [1.5]
    zn, eta = orc.cdcq_tables(2, None, th, y0, 2.0, 4, 5)
    x = hermite_e.hermegauss(5)[0]
    for i in range(4):
        t = 0.5 * (i + 1)
        mean = math.exp(-t) * 1.5 + 0.5 * (1 - math.exp(-t))
        sd = 0.3 * math.sqrt((1 - math.exp(-2 * t)) / 2)
        assert np.allclose(zn[0, i], mean + sd * x, rtol=1e-12)
    # G_{i+1}(eta[k][j]) are the conditional points at the nodes of t_i (exact OU map)
    zc, C = orc.cdc_tables(2, None, th, y0, 2.0, 4, 5)
    for i in range(4):
        got = np.array([[orc.cdcq_G(zn[0, i], eta[0, i, k, j]) for j in range(5)] for k in range(5)])
        assert np.allclose(got, C[0, i], rtol=1e-10, atol=1e-12)
