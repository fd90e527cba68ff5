"""Pins of the oracle's random numbers, Gauss-Hermite points and Lagrange map.

* Philox4x32-10 against the published known-answer vectors (tests/golden).
* The Box-Muller wiring: the radius of each normal pair equals
  sqrt(-2 ln u) of the pair's first raw word; sample moments and a KS test.
* Gauss-Hermite (probabilists'): closed-form roots for m=5, numpy's
  hermegauss, exact normal moments up to degree 2m-1 and failure at 2m.
* Quantile ranks: the inverse empirical CDF at Phi(x_j), via scipy.
* Lagrange map g_m (the 7L interpolation): g_m(x_j) = y_j, reproduces every
  polynomial of degree <= m-1 (compared with numpy.polyfit), partition of unity.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import hermite_e
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = orc.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == out


def test_box_muller_wiring(orc):
    seed, tag, s, q = 0x123456789ABCDEF, 0, 7, 11
    for blk in range(3):
        w = orc.philox4x32_10([blk, q, s, tag], [seed & 0xFFFFFFFF, seed >> 32])
        z = orc.normals(seed, tag, s, q, 4 * blk, 4)
        for pair in range(2):
            u = ((int(w[2 * pair]) >> 9) + 0.5) / 2.0 ** 23
            r2 = -2.0 * math.log(u)
            assert z[2 * pair] ** 2 + z[2 * pair + 1] ** 2 == pytest.approx(r2, rel=1e-13)
            ua = ((int(w[2 * pair + 1]) >> 9) + 0.5) / 2.0 ** 23
            ang = math.atan2(z[2 * pair + 1], z[2 * pair]) % (2 * math.pi)
            assert ang == pytest.approx(2 * math.pi * ua, abs=1e-12)


def test_normal_statistics(orc):
    z = np.concatenate([orc.normals(1, 0, 0, q, 0, 64) for q in range(4000)])
    n = z.size
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1) < 4 * math.sqrt(2.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # different tags / sets / paths give different streams
    a = orc.normals(1, 0, 0, 0, 0, 8)
    b = orc.normals(1, 1, 0, 0, 0, 8)
    c = orc.normals(1, 0, 1, 0, 0, 8)
    assert not np.allclose(a, b) and not np.allclose(a, c)


def test_gh_closed_form_m5(orc):
    x, w = orc.gauss_hermite(5)
    r1, r2 = math.sqrt(5 - math.sqrt(10)), math.sqrt(5 + math.sqrt(10))
    assert np.allclose(x, [-r2, -r1, 0.0, r1, r2], rtol=0, atol=1e-14)
    assert x[2] == 0.0
    assert w.sum() == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7, 8])
def test_gh_vs_numpy_and_moments(orc, m):
    x, w = orc.gauss_hermite(m)
    xr, wr = hermite_e.hermegauss(m)
    assert np.allclose(x, xr, atol=1e-13)
    assert np.allclose(w, wr / wr.sum(), atol=1e-14)
    assert np.all(np.diff(x) > 0)
    assert np.allclose(x, -x[::-1], atol=0)
    # E[X^k] for X ~ N(0,1): 0 for odd k, (k-1)!! for even k; exact up to 2m-1.
    def moment(k):
        return 0.0 if k % 2 else float(np.prod(np.arange(k - 1, 0, -2))) if k else 1.0
    for k in range(2 * m):
        scale = np.dot(w, np.abs(x) ** k)      # size of the terms that cancel
        assert np.dot(w, x ** k) == pytest.approx(moment(k), rel=1e-12, abs=1e-14 * scale)
    assert abs(np.dot(w, x ** (2 * m)) - moment(2 * m)) > 1e-3


@pytest.mark.parametrize("m,n", [(5, 100000), (7, 100000), (7, 10000), (3, 17), (8, 1)])
def test_quantile_ranks(orc, m, n):
    xr, _ = hermite_e.hermegauss(m)
    want = np.clip(np.ceil(n * stats.norm.cdf(xr)).astype(np.int64) - 1, 0, n - 1)
    assert np.array_equal(orc.quantile_ranks(m, n), want)


@pytest.mark.parametrize("m", [2, 5, 7, 8])
def test_lagrange_identities(orc, m):
    rng = np.random.default_rng(m)
    x, _ = orc.gauss_hermite(m)
    y = rng.standard_normal(m)
    for j in range(m):
        assert orc.lagrange(x, y, x[j]) == pytest.approx(y[j], abs=1e-13)
    # reproduces a random polynomial of degree m-1 anywhere (incl. extrapolation)
    c = rng.standard_normal(m)
    yp = np.polyval(c, x)
    for X in np.linspace(-5.5, 5.5, 23):
        assert orc.lagrange(x, yp, X) == pytest.approx(np.polyval(c, X), rel=1e-10, abs=1e-10)
    # interpolant equals numpy's polynomial fit through the points
    cf = np.polyfit(x, y, m - 1)
    for X in (-3.3, -0.7, 0.1, 2.9):
        assert orc.lagrange(x, y, X) == pytest.approx(np.polyval(cf, X), rel=1e-9, abs=1e-9)
    # partition of unity
    for X in (-4.0, 0.3, 1.7):
        assert orc.lagrange(x, np.ones(m), X) == pytest.approx(1.0, abs=1e-12)
