"""GPU tests of the batched-theta path: thousands of parameter sets with uneven path
counts in one persistent launch, replayed from a captured CUDA graph.

* A set's paths do not depend on the other sets: the batched call and a call in which
  every other set is empty give bit-identical Y_T for that set (same set index, so the
  same normals; different tile composition and grid), in both network forms.
* A captured CUDA graph replays to bit-identical outputs and per-set moments.
* The CIR batched workload's shape (4096 sets, log-uniform counts) against the FP64
  oracle on sampled paths of sampled sets, including the smallest and largest sets.
* Degenerate batches: every set empty (nothing to do, status clean, means 0), one path.
* Maximum sizes: a set of 2^31 + 129 paths (indices past int32) in both forms, and
  SL_MAX_SETS = 2^24 parameter sets in one launch.
"""
import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W
from tests.helpers import flat_sets, gate, max_abs_normals, rel_err

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _run(sl, net, th, y0, off, T, n_steps, m, seed, moments=False):
    total = int(off[-1])
    n_sets = len(off) - 1
    yt = torch.full((max(total, 1),), float("nan"), dtype=torch.float32, device="cuda")
    mean = torch.full((n_sets,), float("nan"), dtype=torch.float64, device="cuda") if moments else None
    ws = sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(th), _dev(y0), _dev(off, torch.int64), T, n_steps,
                                          m, seed, out_YT=yt, out_mean=mean)
    torch.cuda.synchronize()
    assert sl.workspace_status(ws) == 0
    return yt.cpu().numpy()[:total], (mean.cpu().numpy() if moments else None)


@pytest.mark.parametrize("prec", [0, 1])
def test_sets_independent_of_batch(sl, orc, prec):
    b = W.cir_batched(n_sets=300, lo_exp=1.0, hi_exp=3.0)
    P = W.xavier_params(5, 7, seed=3)
    net = sl.make_net(_dev(P), 5, 7, prec=prec)
    off = b["offsets"]
    full, _ = _run(sl, net, b["theta"], b["Y0"], off, 4.0, 12, 7, 9)
    counts = np.diff(off)
    for s in (0, 1, 137, 299, int(np.argmax(counts)), int(np.argmin(counts))):
        only = np.zeros_like(counts)
        only[s] = counts[s]
        off_s = W.offsets_from_counts(only)
        got, _ = _run(sl, net, b["theta"], b["Y0"], off_s, 4.0, 12, 7, 9)
        assert np.array_equal(got, full[off[s]:off[s + 1]]), s


def test_cuda_graph_replay(sl, orc):
    b = W.cir_batched(n_sets=4096, lo_exp=1.0, hi_exp=2.5)
    P = W.xavier_params(5, 7, seed=4)
    net = sl.make_net(_dev(P), 5, 7, prec=sl.PREC_BF16)
    total = int(b["offsets"][-1])
    th, y0, off = _dev(b["theta"]), _dev(b["Y0"]), _dev(b["offsets"], torch.int64)
    yt = torch.empty(total, dtype=torch.float32, device="cuda")
    mean = torch.empty(4096, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    ws = torch.empty(sl.simulate_workspace_size(total, 4096), dtype=torch.uint8, device="cuda")
    run = lambda: sl.seven_league_simulate_batched(sl.MODEL_MLP, net, th, y0, off, b["T"], b["n_steps"], 7,
                                                   b["seed"], out_YT=yt, out_mean=mean, out_var=var, ws=ws,
                                                   total_paths=total)
    run()
    torch.cuda.synchronize()
    ref = (yt.clone(), mean.clone(), var.clone())
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run()
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        run()
    for t in (yt, mean, var):
        t.fill_(float("nan"))
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert sl.workspace_status(ws) == 0
    assert torch.equal(yt, ref[0]) and torch.equal(mean, ref[1]) and torch.equal(var, ref[2])


def test_cir_batched_vs_oracle_sampled(sl, orc):
    """4096 sets (path counts 10..1000), 32 steps of dt = 0.25: sampled paths of sampled sets."""
    b = W.cir_batched(n_sets=4096, lo_exp=1.0, hi_exp=3.0)
    P = W.xavier_params(5, 7, seed=5)
    net = sl.make_net(_dev(P), 5, 7, prec=sl.PREC_BF16)
    off = b["offsets"]
    yt, mean = _run(sl, net, b["theta"], b["Y0"], off, b["T"], b["n_steps"], 7, b["seed"], moments=True)
    counts = np.diff(off)
    rng = np.random.default_rng(0)
    sets = np.unique(np.concatenate([rng.integers(0, 4096, 40), [int(np.argmax(counts)), int(np.argmin(counts))]]))
    idx = np.concatenate([np.arange(off[s], off[s + 1]) for s in sets])
    want = orc.seven_league_paths(0, W.bf16_round(P).astype(np.float64), b["theta"], b["Y0"], off, b["T"],
                                  b["n_steps"], 7, b["seed"], d_in=5, idx=idx)
    st, q = flat_sets(off, idx)
    mx = max_abs_normals(orc, b["seed"], 0, st, q, b["n_steps"])
    ok, *info = gate(rel_err(yt[idx], want, 0.1), mx, 2e-3)
    assert ok, info
    for s in sets:
        seg = yt[off[s]:off[s + 1]].astype(np.float64)
        assert mean[s] == pytest.approx(seg.mean(), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("prec", [0, 1])
def test_degenerate_batches(sl, orc, prec):
    P = W.xavier_params(4, 7, seed=6)
    net = sl.make_net(_dev(P), 4, 7, prec=prec)
    th = W.gbm_online_thetas(5)
    off = W.offsets_from_counts([0, 0, 0, 0, 0])
    yt, mean = _run(sl, net, th, np.ones(5, np.float32), off, 1.0, 4, 7, 1, moments=True)
    assert yt.size == 0 and np.all(mean == 0)
    off = W.offsets_from_counts([0, 0, 1, 0, 0])
    yt, mean = _run(sl, net, th, np.ones(5, np.float32), off, 1.0, 4, 7, 1, moments=True)
    want = orc.seven_league_paths(0, (W.bf16_round(P) if prec else P).astype(np.float64), th, np.ones(5), off, 1.0,
                                  4, 7, 1, d_in=4)
    assert abs(yt[0] - want[0]) <= (2e-3 if prec else 1e-5) * (abs(want[0]) + 1.0)
    assert mean[2] == yt[0] and mean[0] == 0


def test_long_horizon_bf16(sl, orc):
    """128 coarse steps in one launch (the time loop stays on chip)."""
    P = W.xavier_params(4, 7, seed=7)
    net = sl.make_net(_dev(P), 4, 7, prec=sl.PREC_BF16)
    th = W.gbm_online_thetas(2)
    off = W.offsets_from_counts([700, 1300])
    yt, _ = _run(sl, net, th, np.ones(2, np.float32), off, 8.0, 128, 7, 3)
    want = orc.seven_league_paths(0, W.bf16_round(P).astype(np.float64), th, np.ones(2), off, 8.0, 128, 7, 3,
                                  d_in=4)
    st, q = flat_sets(off, np.arange(2000))
    mx = max_abs_normals(orc, 3, 0, st, q, 128)
    ok, *info = gate(rel_err(yt, want, 1.0), mx, 2e-3)
    assert ok, info


@pytest.mark.parametrize("prec", [0, 1])
def test_more_than_2_31_paths(sl, orc, prec):
    """One set of 2^31 + 129 paths (flat and in-set path indices past the int32 range), 1 step:
    sampled paths including the last ones agree with the oracle; the set mean is finite."""
    n = (1 << 31) + 129
    P = W.xavier_params(4, 7, seed=8)
    net = sl.make_net(_dev(P), 4, 7, prec=prec)
    th = W.gbm_online_thetas(1)
    off = W.offsets_from_counts([n])
    yt = torch.empty(n, dtype=torch.float32, device="cuda")
    mean = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(th), _dev([1.0]), _dev(off, torch.int64), 1.0, 1,
                                          7, 2, out_YT=yt, out_mean=mean)
    assert sl.workspace_status(ws) == 0
    idx = np.concatenate([np.arange(0, 64), np.arange((1 << 31) - 64, (1 << 31) + 64), np.arange(n - 64, n)])
    Pw = (W.bf16_round(P) if prec else P).astype(np.float64)
    want = orc.seven_league_paths(0, Pw, th, [1.0], off, 1.0, 1, 7, 2, d_in=4, idx=idx)
    got = yt[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    assert np.all(rel_err(got, want, 1.0) <= (2e-3 if prec else 1e-5))
    assert np.isfinite(mean.item())
    del yt


def test_max_sets(sl, orc):
    """SL_MAX_SETS (2^24) parameter sets with 0 or 1 path each, 2 steps, BF16 form."""
    n_sets = 1 << 24
    rng = np.random.default_rng(9)
    counts = rng.integers(0, 2, n_sets)
    off = W.offsets_from_counts(counts)
    th = rng.uniform([0.0, 0.1], [0.2, 0.5], (n_sets, 2)).astype(np.float32)
    P = W.xavier_params(4, 7, seed=9)
    net = sl.make_net(_dev(P), 4, 7, prec=sl.PREC_BF16)
    total = int(off[-1])
    yt = torch.empty(total, dtype=torch.float32, device="cuda")
    mean = torch.empty(n_sets, dtype=torch.float64, device="cuda")
    ws = sl.seven_league_simulate_batched(sl.MODEL_MLP, net, _dev(th), _dev(np.ones(n_sets)), _dev(off, torch.int64),
                                          1.0, 2, 7, 4, out_YT=yt, out_mean=mean)
    assert sl.workspace_status(ws) == 0
    sets = np.concatenate([np.nonzero(counts)[0][:50], np.nonzero(counts)[0][-50:]])
    idx = off[sets]
    want = orc.seven_league_paths(0, W.bf16_round(P).astype(np.float64), th, np.ones(n_sets), off, 1.0, 2, 7, 4,
                                  d_in=4, idx=idx)
    got = yt.cpu().numpy()[idx]
    assert np.all(rel_err(got, want, 1.0) <= 2e-3)
    m = mean.cpu().numpy()
    assert np.array_equal(m[sets], got.astype(np.float64)) and np.all(m[counts == 0] == 0)
