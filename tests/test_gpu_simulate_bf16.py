"""GPU parity of the BF16 tcgen05 7L sampler against the FP64 oracle.

The oracle runs with the same BF16-valued weights and biases (rounded to
nearest, ties to even), so the difference measures the tensor-core form's own
arithmetic: hi+lo BF16 activations, FP32 accumulation, FP32 state.
Tolerance: 2e-3 on |a - b| / (|b| + Y0) per path, gated on paths whose normals
stay within |X| <= 4 plus the 99.99th percentile over all paths.
"""
import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W
from tests.helpers import flat_sets, gate, max_abs_normals, rel_err, with_biases

pytestmark = pytest.mark.gpu
TOL = 2e-3


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _sim(sl, P, d_in, m, theta, Y0, offsets, T, n_steps, seed, prec, grid=False):
    net = sl.make_net(_dev(P), d_in, m, prec=prec)
    total = int(offsets[-1])
    yt = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    gr = torch.empty((n_steps + 1, total), dtype=torch.float32, device="cuda") if grid else None
    mean = torch.empty(len(offsets) - 1, dtype=torch.float64, device="cuda")
    ws = sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(theta), _dev(Y0),
                                          _dev(offsets, torch.int64), T, n_steps, m, seed,
                                          out_YT=yt, out_grid=gr, out_mean=mean)
    bits = sl.workspace_status(ws)
    assert bits == 0, bits
    out = (yt.cpu().numpy(), mean.cpu().numpy())
    return out + ((gr.cpu().numpy(),) if grid else ())


def _oracle(orc, P, d_in, m, theta, Y0, offsets, T, n_steps, seed, idx=None):
    Pb = W.bf16_round(P).astype(np.float64)
    return orc.seven_league_paths(0, Pb, theta, Y0, offsets, T, n_steps, m, seed, d_in=d_in, idx=idx)


def _check(orc, got, want, offsets, seed, n_steps, idx=None, tol=TOL):
    idx = np.arange(len(want)) if idx is None else idx
    s, q = flat_sets(offsets, idx)
    err = rel_err(got, want, 1.0)
    mx = max_abs_normals(orc, seed, 0, s, q, n_steps)
    ok, max_in, p, max_all = gate(err, mx, tol)
    assert ok, (max_in, p, max_all)
    return max_in, p, max_all


def test_tiny_one_tile(sl, orc):
    """A single partial tile (37 paths), one step: the smallest launch."""
    P = W.xavier_params(3, 5, seed=0)
    th = np.array([[0.3]], np.float32)
    off = W.offsets_from_counts([37])
    yt, _ = _sim(sl, P, 3, 5, th, [1.0], off, 1.0, 1, 1, sl.PREC_BF16)
    want = _oracle(orc, P, 3, 5, th, [1.0], off, 1.0, 1, 1)
    assert np.all(np.isfinite(yt))
    _check(orc, yt, want, off, 1, 1)


def test_gbm_small(sl, orc):
    w = W.gbm_small()
    yt, _ = _sim(sl, w["params"], 3, 5, w["theta"], w["Y0"], w["offsets"], w["T"], w["n_steps"],
                 w["seed"], sl.PREC_BF16)
    want = _oracle(orc, w["params"], 3, 5, w["theta"], w["Y0"], w["offsets"], w["T"], w["n_steps"], w["seed"])
    _check(orc, yt, want, w["offsets"], w["seed"], w["n_steps"])


@pytest.mark.parametrize("m,d_in", [(2, 3), (5, 4), (7, 4), (7, 5), (8, 7), (3, 2), (6, 6)])
def test_ragged_batched_grid(sl, orc, m, d_in):
    P = W.xavier_params(d_in, m, seed=m + d_in)
    rng = np.random.default_rng(m)
    n_sets = 6
    th = rng.uniform(0.05, 0.4, size=(n_sets, d_in - 2)).astype(np.float32)
    counts = [0, 129, 1, 0, 5000, 383]
    off = W.offsets_from_counts(counts)
    y0 = rng.uniform(0.5, 1.5, n_sets).astype(np.float32)
    yt, mean, grid = _sim(sl, P, d_in, m, th, y0, off, 1.5, 6, 3, sl.PREC_BF16, grid=True)
    want = _oracle(orc, P, d_in, m, th, y0, off, 1.5, 6, 3)
    _check(orc, yt, want, off, 3, 6)
    assert np.array_equal(grid[-1], yt)
    for s, c in enumerate(counts):
        if c:
            assert mean[s] == pytest.approx(yt[off[s]:off[s + 1]].astype(np.float64).mean(), rel=1e-12)


def _set_cfg(sl, slots, tpw):
    sl.tc_set_pipeline(1)
    sl.tc_set_slots(slots)
    sl.tc_set_pipeline(tpw)


@pytest.mark.parametrize("slots,tpw", [(4, 2), (2, 2), (4, 1), (3, 1), (2, 1)])
def test_launch_configs_agree(sl, orc, slots, tpw):
    """Per-path results do not depend on tiles in flight or the pipeline shape: the
    same arithmetic on the same inputs, identical up to FP32 rounding (different
    kernel instantiations may contract or schedule a few operations differently)."""
    P = W.xavier_params(4, 7, seed=1)
    th = W.gbm_online_thetas(3)
    off = W.offsets_from_counts([10000, 777, 20001])
    old = (sl.tc_get_slots(), sl.tc_get_pipeline())
    try:
        _set_cfg(sl, 4, 1)
        ref, _ = _sim(sl, P, 4, 7, th, np.ones(3, np.float32), off, 2.0, 16, 5, sl.PREC_BF16)
        _set_cfg(sl, slots, tpw)
        got, _ = _sim(sl, P, 4, 7, th, np.ones(3, np.float32), off, 2.0, 16, 5, sl.PREC_BF16)
    finally:
        _set_cfg(sl, *old)
    assert np.all(rel_err(got, ref, 1.0) <= 1e-6)
    assert np.mean(got == ref) > 0.999
    if (slots, tpw) == (4, 1):
        idx = np.arange(0, len(ref), 7)
        want = _oracle(orc, P, 4, 7, th, np.ones(3), off, 2.0, 16, 5, idx=idx)
        _check(orc, ref[idx], want, off, 5, 16, idx=idx)


def test_bf16_vs_fp32_same_paths(sl, orc):
    P = W.xavier_params(4, 7, seed=2)
    th = W.gbm_online_thetas(4)
    off = W.offsets_from_counts([3000] * 4)
    a, _ = _sim(sl, P, 4, 7, th, np.ones(4, np.float32), off, 2.0, 16, 9, sl.PREC_BF16)
    b, _ = _sim(sl, W.bf16_round(P), 4, 7, th, np.ones(4, np.float32), off, 2.0, 16, 9, sl.PREC_FP32)
    # both forms on the same (BF16-valued) weights and normals agree to the BF16 tolerance
    err = rel_err(a, b, 1.0)
    assert np.percentile(err, 99.99) <= TOL


def test_full_size_gbm_online_sampled(sl, orc):
    w = W.gbm_online()
    off = w["offsets"]
    yt, mean = _sim(sl, w["params"], 4, 7, w["theta"], w["Y0"], off, w["T"], w["n_steps"], w["seed"],
                    sl.PREC_BF16)
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([rng.integers(0, off[-1], 3000), off[1:-1] - 1, off[:-1], [off[-1] - 1]]))
    want = _oracle(orc, w["params"], 4, 7, w["theta"], w["Y0"], off, w["T"], w["n_steps"], w["seed"], idx=idx)
    _check(orc, yt[idx], want, off, w["seed"], w["n_steps"], idx=idx)
    assert np.all(np.isfinite(yt))


@pytest.mark.parametrize("slots", [4, 3, 2])
def test_softplus(sl, orc, slots):
    """Softplus (the paper's activation) in the tensor-core form: log(1 + e^z) on the fast
    exponent/logarithm unit, then the same BF16 hi + lo split; against the FP64 oracle's
    Softplus network with the same BF16 weights."""
    P = W.xavier_params(5, 7, seed=12)
    th = np.random.default_rng(3).uniform(0.05, 0.4, (3, 3)).astype(np.float32)
    off = W.offsets_from_counts([3000, 129, 4000])
    y0 = np.array([1.0, 0.5, 1.5], np.float32)
    old = (sl.tc_get_slots(), sl.tc_get_pipeline())
    try:
        _set_cfg(sl, slots, 1)
        net = sl.make_net(_dev(P), 5, 7, act=sl.ACT_SOFTPLUS, prec=sl.PREC_BF16)
        total = int(off[-1])
        yt = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
        ws = sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(th), _dev(y0), _dev(off, torch.int64), 2.0, 16,
                                              7, 4, out_YT=yt)
        assert sl.workspace_status(ws) == 0
    finally:
        _set_cfg(sl, *old)
    want = orc.seven_league_paths(0, W.bf16_round(P).astype(np.float64), th, y0, off, 2.0, 16, 7, 4, d_in=5,
                                  act=orc.ACT_SOFTPLUS)
    _check(orc, yt.cpu().numpy(), want, off, 4, 16)


def _with_biases(P, d_in, m, scale, seed):
    return with_biases(P, W.layer_shapes(d_in, m), scale, seed)


@pytest.mark.parametrize("act", ["relu", "softplus"])
@pytest.mark.parametrize("m,d_in", [(2, 3), (5, 4), (8, 7), (3, 2), (6, 6)])
def test_biases_every_shape(sl, orc, act, m, d_in):
    """Nonzero biases (up to 4 in magnitude) in every layer, for every feature count: the
    layer-1 bias unit sits in feature column d_in (the last one for d_in = 7) and the hidden and
    output biases on the hidden A row's bias unit.  (The Softplus form's bias unit is log2(e) as
    a BF16 hi + lo pair; without the lo entry every bias would be scaled by 1.0018, which the
    gate catches for three of these five shapes, checked with the oracle:
    test_bias_chain_constant_features catches it for every network.)"""
    P = _with_biases(W.xavier_params(d_in, m, seed=40 + m + d_in), d_in, m, 4.0, seed=m * 10 + d_in)
    rng = np.random.default_rng(m + d_in)
    n_sets = 3
    th = rng.uniform(0.05, 0.4, size=(n_sets, d_in - 2)).astype(np.float32)
    off = W.offsets_from_counts([1500, 131, 2200])
    y0 = np.array([1.0, 0.6, 1.4], np.float32)
    a = sl.ACT_SOFTPLUS if act == "softplus" else sl.ACT_RELU
    net = sl.make_net(_dev(P), d_in, m, act=a, prec=sl.PREC_BF16)
    total = int(off[-1])
    yt = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    ws = sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(th), _dev(y0), _dev(off, torch.int64), 1.5, 8,
                                          m, 5, out_YT=yt)
    assert sl.workspace_status(ws) == 0
    want = orc.seven_league_paths(0, W.bf16_round(P).astype(np.float64), th, y0, off, 1.5, 8, m, 5, d_in=d_in,
                                  act=orc.ACT_SOFTPLUS if act == "softplus" else orc.ACT_RELU)
    got = yt.cpu().numpy()
    assert np.all(np.isfinite(got))
    _check(orc, got, want, off, 5, 8)


@pytest.mark.parametrize("act", ["relu", "softplus"])
@pytest.mark.parametrize("seed", [0, 1])
def test_bias_chain_constant_features(sl, orc, act, seed):
    """W1 = 0 and biases up to 4 in every layer: every path gets the same collocation points (the
    chain of biases and hidden weights), so the per-path error is the hi + lo split's rounding of
    constant activations and the gate can be 1e-4.  Checked with the oracle: scaling every bias
    by hi / log2(e) (a Softplus bias unit that lost its lo entry) moves the paths by ~2e-3."""
    d_in, m = 4, 7
    P = _with_biases(W.xavier_params(d_in, m, seed=60 + seed), d_in, m, 4.0, seed=70 + seed)
    P[:50 * d_in] = 0.0
    th = W.gbm_online_thetas(2)
    off = W.offsets_from_counts([2000, 777])
    y0 = np.array([1.0, 0.7], np.float32)
    a = sl.ACT_SOFTPLUS if act == "softplus" else sl.ACT_RELU
    net = sl.make_net(_dev(P), d_in, m, act=a, prec=sl.PREC_BF16)
    total = int(off[-1])
    yt = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    ws = sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(th), _dev(y0), _dev(off, torch.int64), 1.0, 4,
                                          m, 9, out_YT=yt)
    assert sl.workspace_status(ws) == 0
    want = orc.seven_league_paths(0, W.bf16_round(P).astype(np.float64), th, y0, off, 1.0, 4, m, 9, d_in=d_in,
                                  act=orc.ACT_SOFTPLUS if act == "softplus" else orc.ACT_RELU)
    _check(orc, yt.cpu().numpy(), want, off, 9, 4, tol=1e-4)
