"""Failure reporting on the GPU, made on the host side (no fault, trap or hang):

* a forced NaN theta makes the paths non-finite: the sampler (both network forms) and the
  adjoint set SL_DEV_NONFINITE and sl_workspace_status reports SL_ERR_DEVICE;
* a segment with a negative length in the quantile select sets SL_DEV_OFFSETS, the bad
  segment's labels are NaN and the other segments are still exact;
* the bounded-wait self-test: a wait on an mbarrier nothing arrives on gives up after about
  a second with SL_DEV_TIMEOUT, and the context stays usable (a sampler call afterwards is
  correct);
* tiny path counts around the 128-path tile (1, 127, 128, 129 paths; 1 and 3 steps) in both
  network forms against the oracle.
"""
import time

import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("form", ["bf16_network", "fp32_exact_gbm"])
def test_nan_theta_flags_nonfinite(sl, orc, form):
    """NaN in theta of set 1.  (The FP32 network form is not used here: its ReLU, fmaxf(z, 0),
    maps a NaN pre-activation to 0, so NaN features need not reach the state; the exact GBM
    map multiplies the state by exp(NaN).)"""
    if form == "bf16_network":
        model, net = sl.MODEL_MLP, sl.make_net(_dev(W.xavier_params(4, 7, seed=1)), 4, 7, prec=sl.PREC_BF16)
    else:
        model, net = sl.MODEL_GBM_EXACT, None
    th = W.gbm_online_thetas(3)
    th[1, 0] = np.nan
    off = W.offsets_from_counts([300, 200, 100])
    yt = torch.empty(600, dtype=torch.float32, device="cuda")
    ws = sl.seven_league_simulate_batched(model, net, _dev(th), _dev(np.ones(3)), _dev(off, torch.int64),
                                          1.0, 4, 7, 1, out_YT=yt)
    assert sl.workspace_status(ws) & sl.SL_DEV_NONFINITE
    y = yt.cpu().numpy()
    assert np.all(np.isnan(y[300:500])) and np.all(np.isfinite(y[:300])) and np.all(np.isfinite(y[500:]))
    with pytest.raises(sl.SLError):
        sl._check(sl.load().sl_workspace_status(sl._ptr(ws), None, None))
    # the adjoint reports it too
    ws_a = torch.empty(sl.adjoint_workspace_size(600, 3, 4, 2, 2), dtype=torch.uint8, device="cuda")
    sl.seven_league_adjoint(model, net, _dev(th), _dev(np.ones(3)), _dev(off, torch.int64), 1.0, 4, 7, 1,
                            -1.0, ckpt_k=2, ws=ws_a)
    assert sl.workspace_status(ws_a) & sl.SL_DEV_NONFINITE


def test_select_negative_segment_flags_offsets(sl, orc):
    rng = np.random.default_rng(0)
    vals = rng.normal(size=40).astype(np.float32)
    seg = np.array([0, 10, 5, 40], dtype=np.int64)     # segment 1 has length -5
    ranks = np.array([0, 2], dtype=np.int64)
    ws = torch.empty(sl.load().sl_select_workspace_size(3, 2), dtype=torch.uint8, device="cuda")
    out = sl.segmented_select(_dev(vals), _dev(seg, torch.int64), ranks, ws=ws)
    assert sl.workspace_status(ws) & sl.SL_DEV_OFFSETS
    o = out.cpu().numpy().reshape(3, 2)
    assert np.all(np.isnan(o[1]))
    assert np.array_equal(o[0], np.sort(vals[0:10])[ranks]) and np.array_equal(o[2], np.sort(vals[5:40])[ranks])


def test_bounded_wait_gives_up(sl, orc):
    t0 = time.time()
    ws = sl.selftest_wait_timeout()
    bits = sl.workspace_status(ws)
    dt = time.time() - t0
    assert bits == sl.SL_DEV_TIMEOUT, bits
    assert 0.5 < dt < 30.0
    # the context is still usable
    P = W.xavier_params(4, 7, seed=2)
    net = sl.make_net(_dev(P), 4, 7, prec=sl.PREC_BF16)
    th = W.gbm_online_thetas(1)
    off = W.offsets_from_counts([500])
    yt = torch.empty(500, dtype=torch.float32, device="cuda")
    ws2 = sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(th), _dev([1.0]), _dev(off, torch.int64), 1.0,
                                           4, 7, 3, out_YT=yt)
    assert sl.workspace_status(ws2) == 0
    want = orc.seven_league_paths(0, W.bf16_round(P).astype(np.float64), th, [1.0], off, 1.0, 4, 7, 3, d_in=4)
    assert np.all(rel_err(yt.cpu().numpy(), want, 1.0) <= 2e-3)


@pytest.mark.parametrize("n", [1, 127, 128, 129])
@pytest.mark.parametrize("n_steps", [1, 3])
def test_tiny_path_counts(sl, orc, n, n_steps):
    P = W.xavier_params(4, 7, seed=3)
    th = W.gbm_online_thetas(1)
    off = W.offsets_from_counts([n])
    for prec, tol in ((sl.PREC_FP32, 1e-5), (sl.PREC_BF16, 2e-3)):
        net = sl.make_net(_dev(P), 4, 7, prec=prec)
        yt = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        ws = sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(th), _dev([1.0]), _dev(off, torch.int64), 1.0,
                                              n_steps, 7, 5, out_YT=yt)
        assert sl.workspace_status(ws) == 0
        Pw = (W.bf16_round(P) if prec == sl.PREC_BF16 else P).astype(np.float64)
        want = orc.seven_league_paths(0, Pw, th, [1.0], off, 1.0, n_steps, 7, 5, d_in=4)
        assert np.all(rel_err(yt.cpu().numpy(), want, 1.0) <= tol), prec
