"""Pins of the oracle's offline stage (Algorithm I step 1): Euler-Maruyama
(Eq. 6.2) paths and the empirical-quantile collocation labels.

* GBM EM: E[Y_{k+1}] = (1 + mu dtau) E[Y_k] and
  E[Y_{k+1}^2] = ((1 + mu dtau)^2 + sigma^2 dtau) E[Y_k^2] hold exactly for
  the scheme, so the sample moments must match within Monte Carlo error.
* OU EM: the scheme is linear-Gaussian, mean and variance follow exact
  recursions, and the terminal law is exactly normal: the quantile labels must
  match mean + sd * x_j within the asymptotic quantile standard error.
* CIR full truncation: with gamma = 0 the scheme is the deterministic Euler
  recursion with closed form ybar + (Y0 - ybar)(1 - kappa dtau)^N; with
  kappa = 0 and paths far from 0, E[Y^2] grows by exactly gamma^2 E[Y] dtau per
  step (the sqrt(Y) diffusion); terminal samples are non-negative.
* Order statistics: equal to numpy's sort on ragged segments (incl. empty
  and length-1 segments and ties).
"""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e
from scipy import stats

from paper_2302_05170_b300 import workloads as W


def test_gbm_em_moments(orc):
    mu, sg, Y0, dt, nf, n = 0.15, 0.4, 1.3, 0.5, 100, 100_000
    yt = orc.em_terminal(0, [[mu, sg]], [Y0], [dt], n, nf, seed=3)[0]
    dtau = dt / nf
    e1 = Y0 * (1 + mu * dtau) ** nf
    e2 = Y0 ** 2 * ((1 + mu * dtau) ** 2 + sg * sg * dtau) ** nf
    se1 = math.sqrt((e2 - e1 * e1) / n)
    assert abs(yt.mean() - e1) < 4 * se1
    se2 = (yt ** 2).std() / math.sqrt(n)
    assert abs((yt ** 2).mean() - e2) < 4 * se2


def test_ou_em_moments_and_labels(orc):
    yb, sg, lam, Y0, dt, nf, n, m = 0.4, 0.3, 1.5, 1.0, 0.8, 100, 100_000, 7
    th = [[yb, sg, lam]]
    yt = orc.em_terminal(1, th, [Y0], [dt], n, nf, seed=4)[0]
    dtau = dt / nf
    mean, var = Y0, 0.0
    for _ in range(nf):
        mean = mean - lam * (mean - yb) * dtau
        var = (1 - lam * dtau) ** 2 * var + sg * sg * dtau
    assert abs(yt.mean() - mean) < 4 * math.sqrt(var / n)
    assert yt.var() == pytest.approx(var, rel=4 * math.sqrt(2.0 / n))
    lab = orc.em_labels(1, th, [Y0], [dt], n, nf, m, seed=4)[0]
    x, _ = hermite_e.hermegauss(m)
    sd = math.sqrt(var)
    q = mean + sd * x
    lev = stats.norm.cdf(x)
    qse = np.sqrt(lev * (1 - lev) / n) / (stats.norm.pdf(x) / sd)
    assert np.all(np.abs(lab - q) < 5 * qse + 1e-12)
    # labels are the order statistics of the same terminal samples
    ranks = orc.quantile_ranks(m, n)
    assert np.array_equal(lab, np.sort(yt)[ranks])


def test_cir_deterministic_limit(orc):
    kappa, ybar, Y0, dt, nf = 1.7, 0.2, 0.45, 0.9, 100
    yt = orc.em_terminal(2, [[kappa, ybar, 0.0]], [Y0], [dt], 5, nf, seed=1)[0]
    want = ybar + (Y0 - ybar) * (1 - kappa * dt / nf) ** nf
    assert np.allclose(yt, want, rtol=1e-13)


def test_cir_diffusion_term(orc):
    gamma, Y0, dt, nf, n = 0.05, 1.0, 0.5, 100, 200_000
    yt = orc.em_terminal(2, [[0.0, 0.1, gamma]], [Y0], [dt], n, nf, seed=2)[0]
    assert yt.min() > 0.5                      # far from the truncation at 0
    e2 = Y0 ** 2 + gamma ** 2 * Y0 * dt        # E[Y] stays Y0 (martingale)
    assert abs(yt.mean() - Y0) < 4 * yt.std() / math.sqrt(n)
    assert abs((yt ** 2).mean() - e2) < 4 * (yt ** 2).std() / math.sqrt(n)
    assert (yt ** 2).mean() - Y0 ** 2 > 0.5 * gamma ** 2 * Y0 * dt


def test_cir_truncation_nonnegative(orc):
    th, yi, dt = W.cir_label_rows(8)
    th[:, 2] = 0.5     # strong volatility: many paths reach 0
    yi[:] = 0.02
    out = orc.em_terminal(2, th, yi, dt, 2000, 100, seed=9)
    assert out.min() >= 0.0 and (out == 0.0).mean() > 0.002


@pytest.mark.parametrize("ties", [False, True])
def test_order_statistics_bruteforce(orc, ties):
    v, off = W.random_segments(40, 300, seed=11, ties=ties)
    ranks = np.array([0, 1, 5, 17, 123, 299])
    got = orc.order_statistics(v, off, ranks)
    for s in range(len(off) - 1):
        seg = np.sort(v[off[s]:off[s + 1]].astype(np.float64))
        for j, r in enumerate(ranks):
            if r < seg.size:
                assert got[s, j] == seg[r]
            else:
                assert np.isnan(got[s, j])


def test_labels_row_offsets(orc):
    th, yi, dt = W.cir_label_rows(5)
    a = orc.em_labels(2, th, yi, dt, 500, 100, 7, seed=2)
    b = orc.em_labels(2, th, yi, dt, 500, 100, 7, seed=2, row0=3, n_rows=2)
    assert np.array_equal(a[3:], b)
    assert np.all(np.diff(a, axis=1) >= 0)
