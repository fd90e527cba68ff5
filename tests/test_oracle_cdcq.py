"""Pins of the oracle's quantile-coordinate 7L-CDC chain (the marginal collocation map
G_i(xi) = sum_k z_k L_k(xi) through the Gauss-Hermite points carries each path as xi; the
conditional points are moved into the next step's coordinate by G_{i+1}^{-1}).

* G interpolates (x_k, z_k) and continues linearly beyond the outer points; where G increases
  (a quantile map) G^{-1} inverts it (G^{-1}(z_k) = x_k, G(G^{-1}(y)) = y inside and outside the
  range); a constant G inverts to 0 and a G that does not increase from its first to its last
  point to NaN.
* Where G wiggles inside a node interval, G^{-1}(y) is the smallest root of G = y in the first
  node interval that brackets y, however close the next crossings lie: a cubic that crosses y
  twice within 1/32 of a node interval, and random wiggling interpolants, against numpy's
  polynomial roots (companion-matrix eigenvalues) and a dense sign scan.
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


def _first_bracket(z, y):
    k = 0
    while k < len(z) - 2 and not (z[k] <= y <= z[k + 1]):
        k += 1
    return k


def _smallest_root_numpy(x, z, y, k):
    """Smallest real root of G - y in [x_k, x_{k+1}] from the companion-matrix eigenvalues of
    the interpolating polynomial (numpy), polished by Newton in FP64."""
    from numpy.polynomial import polynomial as Pn
    c = Pn.polyfit(x, z, len(x) - 1)
    c[0] -= y
    r = Pn.polyroots(c)
    r = r[np.abs(r.imag) < 1e-7].real
    r = r[(r >= x[k] - 1e-9) & (r <= x[k + 1] + 1e-9)]
    t = float(r.min())
    dc = Pn.polyder(c)
    for _ in range(3):
        t -= Pn.polyval(t, c) / Pn.polyval(t, dc)
    return t


def test_inverse_takes_the_first_of_two_close_crossings(orc):
    """G(xi) = y* + (xi - r1)(xi - r2)(xi - r3) through 4 Gauss-Hermite points: r1 and r2 lie in
    the same 1/32 of the node interval [x_1, x_2], so G exceeds y* only between them and a
    scan of that interval at 32 steps sees G < y* at every point before r3."""
    x = hermite_e.hermegauss(4)[0]
    r1, r2, r3, ys = 0.10, 0.135, 0.62, 20.0
    z = ys + (x - r1) * (x - r2) * (x - r3)
    assert z[0] < z[1] < ys < z[2] < z[3]
    h = (x[2] - x[1]) / 32
    c1, c2 = np.floor((r1 - x[1]) / h), np.floor((r2 - x[1]) / h)
    assert c1 == c2                                 # both crossings inside one cell of the scan
    scan = [orc.cdcq_G(z, x[1] + c * h) for c in range(33)]
    assert all(v < ys for v in scan[: int(np.ceil((r3 - x[1]) / h))])
    got = orc.cdcq_Ginv(z, ys)
    assert got == pytest.approx(r1, abs=1e-12)
    assert got == pytest.approx(_smallest_root_numpy(x, z, ys, 1), abs=1e-12)
    # just above the bump's top the first crossing is r3's; just below r1's level, r1's
    crit = np.roots(np.polyder(np.poly([r1, r2, r3])))
    top = ys + float(np.polyval(np.poly([r1, r2, r3]), crit[(crit > r1) & (crit < r2)][0]))
    assert orc.cdcq_Ginv(z, top + 1e-9) > r2
    assert orc.cdcq_Ginv(z, ys - 1e-9) < r1


@pytest.mark.parametrize("m", [4, 5, 7, 8])
def test_inverse_of_wiggling_maps(orc, m):
    """Random interpolants that increase from the first to the last node but wiggle between:
    G^{-1}(y) is numpy's smallest root in the first bracketing interval, G(G^{-1}(y)) = y, and a
    dense scan finds no crossing before it."""
    from numpy.polynomial import polynomial as Pn
    x = hermite_e.hermegauss(m)[0]
    rng = np.random.default_rng(500 + m)
    n_wiggly = 0
    for trial in range(60):
        z = np.cumsum(rng.uniform(-0.4, 1.0, size=m)) + rng.normal(size=m) * 0.3
        if not z[-1] > z[0]:
            continue
        c = Pn.polyfit(x, z, m - 1)
        for y in rng.uniform(z[0], z[-1], size=8):
            k = _first_bracket(z, y)
            got = orc.cdcq_Ginv(z, y)
            assert x[k] <= got <= x[k + 1]
            assert orc.cdcq_G(z, got) == pytest.approx(y, abs=1e-10 * (1 + abs(y)))
            assert got == pytest.approx(_smallest_root_numpy(x, z, y, k), abs=1e-8)
            g = Pn.polyval(np.linspace(x[k], got, 4001)[:-1], c)
            assert np.all(g < y + 1e-12)
            n_wiggly += int(np.any(np.diff(Pn.polyval(np.linspace(x[k], x[k + 1], 400), c)) < 0))
    assert n_wiggly > 20                            # the sample does exercise non-monotone intervals


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
