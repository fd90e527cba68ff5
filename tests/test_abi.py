"""CPU checks of the C ABI (no GPU needed, no kernel launched).

* The library builds for sm_103a, loads, and exports every function that
  include/sevenleague.h declares; the binding's symbol list matches.
* Host-side numerics: Golub-Welsch Gauss-Hermite points against the closed
  form for m = 5, against numpy's hermegauss and the exact normal moments;
  first-form barycentric weights against their definition via numpy.poly;
  quantile ranks against scipy.
* Host-side argument checks return the documented status codes before any
  device work is enqueued.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest
from numpy.polynomial import hermite_e
from scipy import stats

import paper_2302_05170_b300 as sl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sl.build()
    return sl.load()


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = mt.group(1)
            if name not in ("if", "sizeof", "defined"):
                names.append(name)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(sl.EXPORTED) == declared


def test_version_and_params(lib):
    assert sl.version() >= 100
    from paper_2302_05170_b300 import workloads as W
    for d_in, m in [(3, 5), (4, 7), (5, 7), (7, 8)]:
        assert sl.n_params(d_in, m) == W.n_params(d_in, m)


def test_gauss_hermite_closed_form(lib):
    x, w, b = sl.gauss_hermite(5)
    r1, r2 = math.sqrt(5 - math.sqrt(10)), math.sqrt(5 + math.sqrt(10))
    assert np.allclose(x, [-r2, -r1, 0, r1, r2], atol=1e-14)
    assert x[2] == 0.0
    assert w.sum() == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("m", range(2, 9))
def test_gauss_hermite_vs_numpy(lib, m):
    x, w, b = sl.gauss_hermite(m)
    xr, wr = hermite_e.hermegauss(m)
    assert np.allclose(x, xr, atol=1e-13)
    assert np.allclose(w, wr / wr.sum(), atol=1e-14)
    for k in range(2 * m):
        want = 0.0 if k % 2 else float(np.prod(np.arange(k - 1, 0, -2))) if k else 1.0
        assert np.dot(w, x ** k) == pytest.approx(want, rel=1e-12, abs=1e-14 * np.dot(w, np.abs(x) ** k))
    # first-form barycentric weights: 1 / l'(x_j), l(x) = prod_k (x - x_k)
    dl = np.polyval(np.polyder(np.poly(xr)), xr)
    assert np.allclose(b, 1.0 / dl, rtol=1e-11)


@pytest.mark.parametrize("m,n", [(5, 100000), (7, 100000), (7, 10000), (2, 3), (8, 1)])
def test_quantile_ranks(lib, m, n):
    xr, _ = hermite_e.hermegauss(m)
    want = np.clip(np.ceil(n * stats.norm.cdf(xr)).astype(np.int64) - 1, 0, n - 1)
    assert np.array_equal(sl.quantile_ranks(m, n), want)


def test_host_argument_checks(lib):
    L = lib
    assert L.sl_gauss_hermite(1, None, None, None) == sl.SL_ERR_UNSUPPORTED
    assert L.sl_gauss_hermite(9, None, None, None) == sl.SL_ERR_UNSUPPORTED
    assert L.sl_quantile_ranks(5, 0, None) == sl.SL_ERR_ARG
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every call below is rejected first
    net = sl.sl_net(0x1000, 3, 5, sl.ACT_RELU, sl.PREC_FP32)
    base = dict(model=sl.MODEL_MLP, net=ctypes.byref(net), theta=fake, p=1, Y0=fake, off=fake,
                n_sets=1, total=10, T=1.0, n_steps=2, m=5, seed=1, yt=fake, grid=None, mean=None,
                var=None, ws=fake, ws_bytes=1 << 20, stream=None)

    def call(**kw):
        a = dict(base, **kw)
        return L.seven_league_simulate_batched(a["model"], a["net"], a["theta"], a["p"], a["Y0"], a["off"],
                                               a["n_sets"], a["total"], a["T"], a["n_steps"], a["m"],
                                               a["seed"], a["yt"], a["grid"], a["mean"], a["var"],
                                               a["ws"], a["ws_bytes"], a["stream"])
    assert call(m=9) == sl.SL_ERR_UNSUPPORTED
    assert call(m=1) == sl.SL_ERR_UNSUPPORTED
    assert call(n_steps=0) == sl.SL_ERR_UNSUPPORTED
    assert call(T=-1.0) == sl.SL_ERR_ARG
    assert call(T=float("nan")) == sl.SL_ERR_ARG
    assert call(model=7) == sl.SL_ERR_ARG
    assert call(p=2) == sl.SL_ERR_ARG                       # d_in != p + 2
    assert call(net=None) == sl.SL_ERR_ARG
    assert call(theta=None) == sl.SL_ERR_ARG
    assert call(off=None) == sl.SL_ERR_ARG
    assert call(n_sets=0) == sl.SL_ERR_ARG
    assert call(total=-5) == sl.SL_ERR_ARG
    assert call(yt=None) == sl.SL_ERR_ARG                   # no output at all
    assert call(ws=None) == sl.SL_ERR_WORKSPACE
    assert call(yt=None, mean=fake, ws_bytes=300) == sl.SL_ERR_WORKSPACE
    assert call(model=sl.MODEL_GBM_EXACT, net=None, p=3) == sl.SL_ERR_ARG
    assert call(model=sl.MODEL_OU_EXACT, net=None, p=2) == sl.SL_ERR_ARG
    bad_m = sl.sl_net(0x1000, 3, 7, sl.ACT_RELU, sl.PREC_FP32)
    assert call(net=ctypes.byref(bad_m)) == sl.SL_ERR_ARG   # net->m != m
    sp = sl.sl_net(0x1000, 3, 5, sl.ACT_SOFTPLUS, sl.PREC_BF16)
    assert call(net=ctypes.byref(sp), ws_bytes=16) == sl.SL_ERR_WORKSPACE   # accepted by the sampler
    wide = sl.sl_net(0x1000, 8, 5, sl.ACT_RELU, sl.PREC_BF16)
    assert call(net=ctypes.byref(wide), p=6) == sl.SL_ERR_UNSUPPORTED
    assert "d_in" in L.sl_last_error_string().decode()
    # adjoint: the BF16 tensor-core form takes ReLU or Softplus networks with d_in <= 7
    def adj(net_, p=1, k=8):
        return L.seven_league_adjoint(sl.MODEL_MLP, ctypes.byref(net_), fake, p, fake, fake, 1, 10, 1.0, 2, 5, 1,
                                      sl.PAYOFF_CALL, 1.0, k, None, None, None, None, None, fake, 16, None)
    assert adj(sp) == sl.SL_ERR_WORKSPACE                     # accepted; 16 bytes are too few
    assert adj(wide, p=6) == sl.SL_ERR_UNSUPPORTED
    assert adj(sl.sl_net(0x1000, 3, 5, sl.ACT_RELU, 7)) == sl.SL_ERR_ARG          # unknown precision
    assert adj(sl.sl_net(0x1000, 3, 5, sl.ACT_RELU, sl.PREC_BF16), k=33) == sl.SL_ERR_UNSUPPORTED
    assert adj(sl.sl_net(0x1000, 3, 5, sl.ACT_RELU, sl.PREC_BF16), k=8) == sl.SL_ERR_WORKSPACE
    # EM / labels / select
    assert L.sl_em_terminal(5, fake, fake, fake, 4, 10, 100, 1, fake, None) == sl.SL_ERR_ARG
    assert L.sl_em_terminal(0, fake, fake, fake, 4, 10, 0, 1, fake, None) == sl.SL_ERR_UNSUPPORTED
    assert L.sl_em_terminal(0, None, fake, fake, 4, 10, 100, 1, fake, None) == sl.SL_ERR_ARG
    assert L.sl_em_terminal(0, fake, fake, fake, 70000, 10, 100, 1, fake, None) == sl.SL_ERR_UNSUPPORTED
    assert L.em_collocation_labels(2, fake, fake, fake, 4, 100, 100, 9, 1, fake, fake, 1 << 20, None) == sl.SL_ERR_UNSUPPORTED
    assert L.em_collocation_labels(2, fake, fake, fake, 4, 100, 100, 7, 1, fake, fake, 100, None) == sl.SL_ERR_WORKSPACE
    r = (ctypes.c_int64 * 2)(0, 5)
    assert L.sl_segmented_select(fake, fake, 3, r, 0, fake, fake, 256, None) == sl.SL_ERR_UNSUPPORTED
    assert L.sl_segmented_select(fake, fake, 3, r, 17, fake, fake, 256, None) == sl.SL_ERR_UNSUPPORTED
    assert L.sl_segmented_select(fake, fake, 3, r, 2, fake, fake, 16, None) == sl.SL_ERR_WORKSPACE
    neg = (ctypes.c_int64 * 2)(0, -1)
    assert L.sl_segmented_select(fake, fake, 3, neg, 2, fake, fake, 256, None) == sl.SL_ERR_ARG


def test_cdc_argument_checks(lib):
    L = lib
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every call below is rejected first
    net = sl.sl_net(0x1000, 3, 5, sl.ACT_RELU, sl.PREC_FP32)
    base = dict(model=sl.MODEL_MLP, net=ctypes.byref(net), mnet=None, space=sl.CDC_QUANTILE, theta=fake, p=1,
                Y0=fake, off=fake,
                n_sets=1, total=10, T=1.0, n_steps=2, m=5, seed=1, yt=fake, grid=None, mean=None,
                var=None, ws=fake, ws_bytes=256, stream=None)

    def call(**kw):
        a = dict(base, **kw)
        return L.seven_league_cdc_simulate_batched(
            a["model"], a["net"], a["mnet"], a["space"], a["theta"], a["p"], a["Y0"], a["off"], a["n_sets"], a["total"],
            a["T"], a["n_steps"], a["m"], a["seed"], a["yt"], a["grid"], a["mean"], a["var"], a["ws"],
            a["ws_bytes"], a["stream"])
    need = sl.cdc_workspace_size(10, 1, 2)
    assert need >= 256 + 2 * 224 * 4
    assert call() == sl.SL_ERR_WORKSPACE                        # 256 bytes hold no tables
    assert call(space=sl.CDC_Y) == sl.SL_ERR_WORKSPACE
    assert call(space=2) == sl.SL_ERR_ARG
    assert call(m=9) == sl.SL_ERR_UNSUPPORTED
    assert call(n_steps=0) == sl.SL_ERR_UNSUPPORTED
    assert call(T=0.0) == sl.SL_ERR_ARG
    assert call(net=None) == sl.SL_ERR_ARG
    assert call(p=2) == sl.SL_ERR_ARG
    bad = sl.sl_net(0x1000, 3, 7, sl.ACT_RELU, sl.PREC_FP32)   # marginal network of another m
    assert call(mnet=ctypes.byref(bad)) == sl.SL_ERR_ARG
    bad_act = sl.sl_net(0x1000, 3, 5, 5, sl.PREC_FP32)
    assert call(mnet=ctypes.byref(bad_act)) == sl.SL_ERR_ARG
    assert call(Y0=None) == sl.SL_ERR_ARG
    assert call(off=None) == sl.SL_ERR_ARG
    assert call(n_sets=0) == sl.SL_ERR_ARG
    assert call(yt=None) == sl.SL_ERR_ARG
    assert call(ws=None) == sl.SL_ERR_WORKSPACE
    assert call(model=sl.MODEL_GBM_EXACT, net=None, p=3) == sl.SL_ERR_ARG
    # with out_YT given the call needs the status word and the tables: 256 + align256(2 * 896)
    assert call(model=sl.MODEL_OU_EXACT, net=None, p=3, ws_bytes=2047) == sl.SL_ERR_WORKSPACE
    assert sl.cdc_workspace_size(10 ** 6, 16, 16) >= 256 + 16 * 16 * 896 + 4 * 10 ** 6


def test_workspace_sizes(lib):
    assert sl.simulate_workspace_size(0, 1) >= 256
    assert sl.simulate_workspace_size(10 ** 6, 16) >= 256 + 4 * 10 ** 6
    assert sl.em_labels_workspace_size(1024, 10 ** 5, 7) >= 256 + 4 * 1024 * 10 ** 5
