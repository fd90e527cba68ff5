"""The range call that one rank of a split batch runs (seven_league_simulate_range), on the GPU.

A batch is cut into contiguous ranges of its flat path list -- ranks of a world of 2, 3 and 8
(sharding.rank_range), a cut inside a set, an empty range, a range of one path -- and each range
runs alone.  Checked against the whole batched call on the same inputs:
* every path's Y_T, and its grid row, is bit for bit the whole call's (BF16 tensor-core form,
  FP32 form, exact GBM map): a path keeps its set and its index within the set, hence its normals;
* the per-range counts are the set sizes cut by the range, and combining the ranges' FP64 means
  and variances in rank order (sharding.combine_moments) gives the whole call's to rounding;
* simulate_sharded in a single process (world 1) is the whole call.
"""
import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import sharding
from paper_2302_05170_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _batch(sl, model, prec):
    counts = [1000, 1, 0, 4097, 2500, 129]
    off = W.offsets_from_counts(counts)
    th = W.gbm_online_thetas(len(counts))
    y0 = np.linspace(0.8, 1.3, len(counts)).astype(np.float32)
    net = None
    if model == sl.MODEL_MLP:
        P = W.xavier_params(4, 7, seed=3)
        net = sl.make_net(_dev(P), 4, 7, prec=prec)
    return net, _dev(th), _dev(y0), _dev(off, torch.int64), off


@pytest.mark.parametrize("model,prec", [(0, 1), (0, 0), (1, 0)])
def test_ranges_reproduce_the_batched_call(sl, model, prec):
    net, th, y0, o, off = _batch(sl, model, prec)
    total, n_sets, T, n_steps, m, seed = int(off[-1]), len(off) - 1, 2.0, 8, 7, 11
    yt = torch.empty(total, device="cuda")
    grid = torch.empty((n_steps + 1, total), device="cuda")
    mean = torch.empty(n_sets, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    ws = sl.seven_league_simulate_batched(model, net, th, y0, o, T, n_steps, m, seed, out_YT=yt, out_grid=grid,
                                          out_mean=mean, out_var=var)
    assert sl.workspace_status(ws) == 0
    whole, wgrid = yt.cpu().numpy(), grid.cpu().numpy()
    cuts = [[(a, b - a) for a, b in zip(c[:-1], c[1:])] for c in
            ([sharding.rank_range(total, w, r)[0] for r in range(w)] + [total] for w in (2, 3, 8))]
    cuts.append([(0, 1500), (1500, 0), (1500, 1), (1501, total - 1501)])     # cut inside set 3, empty, one path
    for ranges in cuts:
        parts = []
        for first, n in ranges:
            y = torch.full((max(n, 1),), float("nan"), device="cuda")
            g = torch.empty((n_steps + 1, max(n, 1)), device="cuda")
            c = torch.empty(n_sets, dtype=torch.int64, device="cuda")
            mu, v = torch.empty_like(mean), torch.empty_like(mean)
            w = sl.seven_league_simulate_range(model, net, th, y0, o, T, n_steps, m, seed, first, n, out_YT=y,
                                               out_grid=g, out_mean=mu, out_var=v, out_count=c)
            assert sl.workspace_status(w) == 0
            assert np.array_equal(y.cpu().numpy()[:n], whole[first:first + n])
            assert np.array_equal(g.cpu().numpy()[:, :n], wgrid[:, first:first + n])
            want_c = np.clip(off[1:] - first, 0, n) - np.clip(off[:-1] - first, 0, n)
            assert np.array_equal(c.cpu().numpy(), want_c)
            parts.append((c.cpu().numpy(), mu.cpu().numpy(), v.cpu().numpy()))
        cc, cm, cv = sharding.combine_moments(*[np.array([p[i] for p in parts]) for i in range(3)])
        assert np.array_equal(cc, np.diff(off))
        assert np.allclose(cm, mean.cpu().numpy(), rtol=1e-12, atol=0)
        assert np.allclose(cv, var.cpu().numpy(), rtol=1e-9, atol=0)


def test_single_process_sharded_call_is_the_batched_call(sl):
    net, th, y0, o, off = _batch(sl, 0, 1)
    total = int(off[-1])
    yt = torch.empty(total, device="cuda")
    mean = torch.empty(len(off) - 1, dtype=torch.float64, device="cuda")
    ws = sl.seven_league_simulate_batched(0, net, th, y0, o, 1.0, 4, 7, 2, out_YT=yt, out_mean=mean)
    ys = torch.empty(total, device="cuda")
    r = sharding.simulate_sharded(0, net, th, y0, o, 1.0, 4, 7, 2, out_YT=ys)
    assert sl.workspace_status(ws) == 0 and sl.workspace_status(r["ws"]) == 0
    assert (r["first"], r["n_paths"]) == (0, total)
    assert np.array_equal(ys.cpu().numpy(), yt.cpu().numpy())
    assert np.allclose(r["mean"], mean.cpu().numpy(), rtol=1e-15, atol=0)


def test_range_argument_errors(sl):
    net, th, y0, o, off = _batch(sl, 0, 1)
    with pytest.raises(sl.SLError) as e:
        sl.seven_league_simulate_range(0, net, th, y0, o, 1.0, 4, 7, 2, -1, 10, out_YT=torch.empty(10, device="cuda"))
    assert e.value.status == sl.SL_ERR_ARG
    with pytest.raises(sl.SLError) as e:
        sl.seven_league_simulate_range(0, net, th, y0, o, 1.0, 4, 7, 2, 0, 10)
    assert e.value.status == sl.SL_ERR_ARG
