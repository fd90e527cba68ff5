"""GPU parity of the FP32 CUDA-core 7L sampler against the FP64 oracle
(Algorithm I, steps 2-8), through the C ABI.

Tolerance: 1e-5 on |a - b| / (|b| + Y0) per path (FP32 arithmetic against
FP64 on the same Philox normals), gated on paths whose normals stay within
|X| <= 4 plus the 99.99th percentile over all paths; path means within
1e-5 relative of the oracle's.  Sizes span many CTAs and a ragged tail.
"""
import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W
from tests.helpers import flat_sets, gate, max_abs_normals, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _run(sl, model, net, theta, Y0, offsets, T, n_steps, m, seed, grid=False, moments=False):
    total = int(offsets[-1])
    yt = torch.empty(total, dtype=torch.float32, device="cuda")
    gr = torch.empty((n_steps + 1, total), dtype=torch.float32, device="cuda") if grid else None
    mean = torch.empty(len(offsets) - 1, dtype=torch.float64, device="cuda") if moments else None
    var = torch.empty_like(mean) if moments else None
    ws = sl.seven_league_simulate_batched(model, net, _dev(theta), _dev(Y0), _dev(offsets, torch.int64),
                                          T, n_steps, m, seed, out_YT=yt, out_grid=gr, out_mean=mean,
                                          out_var=var)
    assert sl.workspace_status(ws) == 0
    torch.cuda.synchronize()
    out = [yt.cpu().numpy()]
    if grid:
        out.append(gr.cpu().numpy())
    if moments:
        out += [mean.cpu().numpy(), var.cpu().numpy()]
    return out


def _check_paths(orc, got, want, offsets, seed, n_steps, scale, tol=TOL, idx=None):
    idx = np.arange(len(want)) if idx is None else idx
    s, q = flat_sets(offsets, idx)
    err = rel_err(got, want, scale)
    mx = max_abs_normals(orc, seed, 0, s, q, n_steps)
    ok, max_in, p, max_all = gate(err, mx, tol)
    assert ok, (max_in, p, max_all)
    return max_in, p, max_all


def test_gbm_small_mlp(sl, orc):
    """Network 3->50x4->5 ReLU, Xavier seed 0, 1e4 paths, 2 steps (GBM mu=.1 sigma=.3 Y0=1 T=1)."""
    w = W.gbm_small()
    P = torch.as_tensor(w["params"], device="cuda")
    net = sl.make_net(P, 3, 5)
    yt, = _run(sl, 0, net, w["theta"], w["Y0"], w["offsets"], w["T"], w["n_steps"], 5, w["seed"])
    want = orc.seven_league_paths(0, w["params"].astype(np.float64), w["theta"], w["Y0"], w["offsets"],
                                  w["T"], w["n_steps"], 5, w["seed"], d_in=3)
    _check_paths(orc, yt, want, w["offsets"], w["seed"], w["n_steps"], 1.0)


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7, 8])
def test_mlp_all_m_batched_ragged(sl, orc, m):
    d_in = 4
    Pn = W.xavier_params(d_in, m, seed=m)
    net = sl.make_net(torch.as_tensor(Pn, device="cuda"), d_in, m)
    th = W.gbm_online_thetas(5, seed=m)
    counts = [0, 1, 257, 0, 3001]            # empty sets, a single path, ragged tails
    off = W.offsets_from_counts(counts)
    y0 = np.array([1.0, 0.7, 1.3, 2.0, 0.5], np.float32)
    yt, grid, mean, var = _run(sl, 0, net, th, y0, off, 2.0, 5, m, 9, grid=True, moments=True)
    want, wgrid = orc.seven_league_paths(0, Pn.astype(np.float64), th, y0, off, 2.0, 5, m, 9, d_in=4,
                                         grid=True)
    _check_paths(orc, yt, want, off, 9, 5, 1.0)
    assert np.allclose(grid.T, wgrid, rtol=1e-4, atol=1e-5)
    assert np.array_equal(grid[-1], yt)
    om, ov = orc.seven_league_moments(0, Pn.astype(np.float64), th, y0, off, 2.0, 5, m, 9, d_in=4)
    for s, c in enumerate(counts):
        if c == 0:
            assert mean[s] == 0 and var[s] == 0
            continue
        assert mean[s] == pytest.approx(om[s], rel=TOL, abs=TOL)
        if c > 1:
            assert var[s] == pytest.approx(ov[s], rel=1e-4, abs=1e-9)
        # FP64 reduction of the GPU's own Y_T
        seg = yt[off[s]:off[s + 1]].astype(np.float64)
        assert mean[s] == pytest.approx(seg.mean(), rel=1e-13)


def test_softplus(sl, orc):
    d_in, m = 4, 7
    Pn = W.xavier_params(d_in, m, seed=3)
    net = sl.make_net(torch.as_tensor(Pn, device="cuda"), d_in, m, act=sl.ACT_SOFTPLUS)
    th = W.gbm_online_thetas(2)
    off = W.offsets_from_counts([700, 1100])
    y0 = np.ones(2, np.float32)
    yt, = _run(sl, 0, net, th, y0, off, 2.0, 4, m, 2)
    want = orc.seven_league_paths(0, Pn.astype(np.float64), th, y0, off, 2.0, 4, m, 2, d_in=4,
                                  act=orc.ACT_SOFTPLUS)
    _check_paths(orc, yt, want, off, 2, 4, 1.0)


@pytest.mark.parametrize("m", [5, 7])
def test_exact_gbm(sl, orc, m):
    th = np.array([[0.1, 0.3], [0.05, 0.45]], np.float32)
    y0 = np.array([1.0, 2.0], np.float32)
    off = W.offsets_from_counts([20000, 13001])
    yt, mean, var = _run(sl, 1, None, th, y0, off, 1.0, 16, m, 4, moments=True)
    want = orc.seven_league_paths(1, None, th, y0, off, 1.0, 16, m, 4)
    _check_paths(orc, yt, want, off, 4, 16, 1.0)
    om, ov = orc.seven_league_moments(1, None, th, y0, off, 1.0, 16, m, 4)
    assert np.allclose(mean, om, rtol=TOL)


def test_exact_ou_pathwise(sl, orc):
    th = np.array([[0.5, 0.4, 1.3]], np.float32)
    off = W.offsets_from_counts([9999])
    yt, = _run(sl, 2, None, th, np.array([2.0], np.float32), off, 3.0, 6, 5, 7)
    want = orc.seven_league_paths(2, None, th, [2.0], off, 3.0, 6, 5, 7)
    _check_paths(orc, yt, want, off, 7, 6, 1.0)


def test_single_set_api_and_determinism(sl, orc):
    w = W.gbm_small(n_paths=5000)
    P = torch.as_tensor(w["params"], device="cuda")
    net = sl.make_net(P, 3, 5)
    out = torch.empty(5000, device="cuda")
    sl.seven_league_simulate(0, _dev(w["theta"][0]), 1.0, 1.0, 2, 5, net, 5000, 1, out)
    a = out.cpu().numpy()
    b, = _run(sl, 0, net, w["theta"], w["Y0"], w["offsets"], 1.0, 2, 5, 1)
    assert np.array_equal(a, b)
    sl.seven_league_simulate(0, _dev(w["theta"][0]), 1.0, 1.0, 2, 5, net, 5000, 1, out)
    assert np.array_equal(out.cpu().numpy(), a)
    # the set's paths do not depend on sets in front of it
    th2 = np.concatenate([np.array([[0.2]], np.float32), w["theta"]])
    off2 = W.offsets_from_counts([333, 5000])
    c, = _run(sl, 0, net, th2, np.array([1.5, 1.0], np.float32), off2, 1.0, 2, 5, 1)
    off3 = W.offsets_from_counts([0, 5000])
    d, = _run(sl, 0, net, th2, np.array([1.5, 1.0], np.float32), off3, 1.0, 2, 5, 1)
    assert np.array_equal(c[333:], d)


def test_full_size_gbm_online_sampled(sl, orc):
    """16 theta x 1e6 paths x 16 steps, m=7: sampled paths vs the oracle path by path."""
    w = W.gbm_online()
    P = torch.as_tensor(w["params"], device="cuda")
    net = sl.make_net(P, 4, 7)
    off = w["offsets"]
    yt, mean, var = _run(sl, 0, net, w["theta"], w["Y0"], off, w["T"], w["n_steps"], 7, w["seed"],
                         moments=True)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([rng.integers(0, off[-1], 3000), off[1:-1] - 1, off[:-1], [off[-1] - 1]]))
    want = orc.seven_league_paths(0, w["params"].astype(np.float64), w["theta"], w["Y0"], off, w["T"],
                                  w["n_steps"], 7, w["seed"], d_in=4, idx=idx)
    _check_paths(orc, yt[idx], want, off, w["seed"], w["n_steps"], 1.0, idx=idx)
    for s in range(16):
        seg = yt[off[s]:off[s + 1]].astype(np.float64)
        assert mean[s] == pytest.approx(seg.mean(), rel=1e-12)
        assert var[s] == pytest.approx(seg.var(ddof=1), rel=1e-9)
