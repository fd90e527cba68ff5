"""GPU parity of the 7L-CDC sampler in the marginal's quantile coordinate (SL_CDC_SPACE_QUANTILE)
against the FP64 oracle, through the C ABI.

A path carries xi (Y = G_i(xi), G_i the marginal collocation map through the Gauss-Hermite
points); per (set, step) the table holds the conditional points moved into the next step's
coordinate, eta = G_{i+1}^{-1}(C), and the monomial coefficients B of their tensor-product
interpolant, so that xi_{i+1} = sum_a xi^a sum_b B[a][b] X^b.  Both interpolations run through
Gauss-Hermite points, so the FP32 path error needs no condition-number scaling: TOL on
|a - b| / (|b| + s) per path, gated like the 7L sampler (paths whose normals stay within
|X| <= 4, plus the 99.99th percentile over all paths).  FP32 tables (eta, B, G) and FP32
Horner evaluations against FP64 on the same normals: a few 1e-7 per step over up to 16 steps.

* Exact OU map: the chain equals the 7L OU chain (oracle and GPU 7L sampler); exact GBM map.
* Networks (ReLU, Softplus, a separate marginal network): the tables -- nodes of t_{i+1},
  G's coefficients and edges, eta against the oracle's, B from the kernel's own eta -- and the
  paths; a network whose marginal points decrease gives NaN paths (SL_DEV_NONFINITE).
* G^{-1} (sl_cdcq_inverse, the table kernel's routine) against the oracle's smallest root in
  the first bracketing node interval: a cubic that crosses y twice within 1/32 of a node
  interval, random wiggling maps (m = 4..8), monotone maps, values at and beyond the nodes,
  coinciding and decreasing nodes; and in the tables, with a hand-built network that puts a
  conditional point on that double crossing.
* Degenerate laws (sigma = 0), ragged and empty sets, one step, batch independence
  (bit-exact), CUDA graph replay, FP64 set moments, the 16 x 1e6 x 16 workload on sampled paths,
  m = 2..8, 2^31 + 129 paths in one set, 2^20 sets.
"""
import math

import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W
from tests.helpers import flat_sets, gate, max_abs_normals, rel_err

pytestmark = pytest.mark.gpu
TOL = 3e-5


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _run(sl, model, net, theta, Y0, offsets, T, n_steps, m, seed, marg=None, grid=False, moments=False, status=0):
    total = int(offsets[-1])
    n_sets = len(offsets) - 1
    yt = torch.full((max(total, 1),), float("nan"), dtype=torch.float32, device="cuda")
    gr = torch.empty((n_steps + 1, total), dtype=torch.float32, device="cuda") if grid else None
    mean = torch.full((n_sets,), float("nan"), dtype=torch.float64, device="cuda") if moments else None
    var = torch.empty_like(mean) if moments else None
    ws = sl.seven_league_cdc_simulate_batched(model, net, _dev(theta), _dev(Y0), _dev(offsets, torch.int64), T,
                                              n_steps, m, seed, marg_net=marg, space=sl.CDC_QUANTILE, out_YT=yt,
                                              out_grid=gr, out_mean=mean, out_var=var)
    assert sl.workspace_status(ws) == status
    out = dict(yt=yt.cpu().numpy()[:total], tab=sl.cdc_tables(ws, n_sets, n_steps).cpu().numpy())
    if grid:
        out["grid"] = gr.cpu().numpy()
    if moments:
        out["mean"], out["var"] = mean.cpu().numpy(), var.cpu().numpy()
    return out


def _check(orc, got, want, offsets, seed, n_steps, scale, idx=None, tol=TOL):
    idx = np.arange(len(want)) if idx is None else idx
    s, q = flat_sets(offsets, idx)
    err = rel_err(got, want, scale)
    ok, *info = gate(err, max_abs_normals(orc, seed, 0, s, q, n_steps), tol)
    print("per-path error (max |X|<=4, p99.99, max):", info)
    assert ok, info


def _gh_monomials(m):
    from numpy.polynomial import hermite_e, polynomial as Pn
    x = hermite_e.hermegauss(m)[0]
    out = np.zeros((m, m))
    for j in range(m):
        c = np.array([1.0])
        for l in range(m):
            if l != j:
                c = Pn.polymul(c, [-x[l], 1.0])
        out[j] = c / np.prod([x[j] - x[l] for l in range(m) if l != j])
    return x, out


def _tables_vs_oracle(tab, zn, eta, m, tol=1e-5):
    """tab: the kernel's tables [n_sets, n_steps, 224]; zn, eta: the oracle's."""
    x, bq = _gh_monomials(m)
    t = tab.astype(np.float64)
    gz = t[..., :m]
    assert np.abs(gz - zn).max() <= tol * np.abs(zn).max()
    ge = t[..., 24:88].reshape(*t.shape[:2], 8, 8)[..., :m, :m]
    assert np.abs(ge - eta).max() <= tol * max(1.0, np.abs(eta).max())
    # G's coefficients and B from the kernel's own nodes and eta (FP64 sums, one rounding)
    Gm = t[..., 8:8 + m]
    assert np.all(np.abs(Gm - gz @ bq) <= 2 ** -20 * (np.abs(gz) @ np.abs(bq)) + 1e-30)
    B = t[..., 88:152].reshape(*t.shape[:2], 8, 8)[..., :m, :m]
    want = np.einsum("ka,...kj,jb->...ab", bq, ge, bq)
    size = np.einsum("ka,...kj,jb->...ab", np.abs(bq), np.abs(ge), np.abs(bq))
    assert np.all(np.abs(B - want) <= 2 ** -19 * size + 1e-12)
    assert np.allclose(t[..., 16], x[0], rtol=1e-7) and np.allclose(t[..., 17], x[-1], rtol=1e-7)
    assert np.allclose(t[..., 18], (gz[..., 1] - gz[..., 0]) / (x[1] - x[0]), rtol=1e-6, atol=1e-12)
    assert np.array_equal(t[..., 20], t[..., 0]) and np.array_equal(t[..., 21], t[..., m - 1])
    # node rows 0, 1, m-2, m-1 as monomials in X (xi beyond the hull): eta[k] @ bq
    for r, k in enumerate((0, 1, m - 2, m - 1)):
        R = t[..., 152 + 8 * r:152 + 8 * r + m]
        want = ge[..., k, :] @ bq
        size = np.abs(ge[..., k, :]) @ np.abs(bq)
        assert np.all(np.abs(R - want) <= 2 ** -19 * size + 1e-12), k
    assert np.allclose(t[..., 22], x[1], rtol=1e-7) and np.allclose(t[..., 23], x[-2], rtol=1e-7)
    assert np.all(t[..., 184:] == 0) and np.all(t[..., m:8] == 0)


@pytest.mark.parametrize("model,theta,Y0,m", [
    (2, [[0.5, 0.3, 1.0], [1.0, 0.45, 0.6]], [1.5, -0.5], 5),
    (2, [[0.2, 0.2, 1.5]], [0.3], 8),
    (1, [[0.1, 0.3], [0.15, 0.5], [0.0, 0.1]], [1.0, 0.7, 3.0], 7),
])
def test_exact_models(sl, orc, model, theta, Y0, m):
    off = W.offsets_from_counts([3000 + 1111 * s for s in range(len(Y0))])
    r = _run(sl, model, None, theta, Y0, off, 2.0, 16, m, 21)
    want = orc.cdcq_paths(model, None, theta, Y0, off, 2.0, 16, m, 21)
    _check(orc, r["yt"], want, off, 21, 16, 1.0)
    zn, eta = orc.cdcq_tables(model, None, theta, Y0, 2.0, 16, m)
    _tables_vs_oracle(r["tab"], zn, eta, m)
    if model == 2:     # the OU chain is the 7L chain: against the GPU's own 7L sampler too
        yt7 = torch.empty(int(off[-1]), device="cuda")
        ws = sl.seven_league_simulate_batched(2, None, _dev(theta), _dev(Y0), _dev(off, torch.int64), 2.0, 16, m, 21,
                                              out_YT=yt7)
        assert sl.workspace_status(ws) == 0
        _check(orc, r["yt"], yt7.cpu().numpy(), off, 21, 16, 1.0)


@pytest.mark.parametrize("act", [0, 1])
def test_network_tables_and_paths(sl, orc, act):
    d_in, m, n_steps = 4, 7, 8
    P = W.near_affine_params(d_in, m, seed=31)
    net = sl.make_net(_dev(P), d_in, m, act=act)
    th = W.gbm_online_thetas(3)
    y0 = [1.0, 0.8, 1.3]
    off = W.offsets_from_counts([2500, 1, 3333])
    r = _run(sl, 0, net, th, y0, off, 2.0, n_steps, m, 8, grid=True)
    zn, eta = orc.cdcq_tables(0, P, th, y0, 2.0, n_steps, m, d_in=d_in, act=act)
    _tables_vs_oracle(r["tab"], zn, eta, m)
    want, g = orc.cdcq_paths(0, P, th, y0, off, 2.0, n_steps, m, 8, d_in=d_in, act=act, grid=True)
    _check(orc, r["yt"], want, off, 8, n_steps, 1.0)
    assert np.array_equal(r["grid"][-1], r["yt"])
    assert np.all(rel_err(r["grid"].T, g, 1.0)[:, 1:].max(axis=1) <= 1e-4)


def test_separate_marginal_network(sl, orc):
    d_in, m = 5, 5
    P, Pm = W.near_affine_params(d_in, m, seed=32), W.near_affine_params(d_in, m, b=0.4, seed=33)
    th, y0 = [[0.5, 0.3, 1.0], [0.2, 0.4, 1.5]], [1.5, 0.0]
    off = W.offsets_from_counts([1500, 900])
    r = _run(sl, 0, sl.make_net(_dev(P), d_in, m), th, y0, off, 1.5, 6, m, 4, marg=sl.make_net(_dev(Pm), d_in, m))
    zn, eta = orc.cdcq_tables(0, P, th, y0, 1.5, 6, m, Pm=Pm, d_in=d_in)
    _tables_vs_oracle(r["tab"], zn, eta, m)
    _check(orc, r["yt"], orc.cdcq_paths(0, P, th, y0, off, 1.5, 6, m, 4, Pm=Pm, d_in=d_in), off, 4, 6, 1.0)


def test_decreasing_marginal_points_give_nan(sl, orc):
    P = W.near_affine_params(4, 7, a=-0.2, b=-0.3, seed=34)    # points decreasing in j
    r = _run(sl, 0, sl.make_net(_dev(P), 4, 7), W.gbm_online_thetas(1), [1.0], W.offsets_from_counts([300]),
             1.0, 4, 7, 2, status=sl.SL_DEV_NONFINITE)
    assert np.all(np.isnan(r["yt"]))


def test_degenerate_law(sl, orc):
    th, y0 = [[0.1, 0.0], [0.2, 0.0]], [1.0, 2.0]
    off = W.offsets_from_counts([300, 200])
    r = _run(sl, 1, None, th, y0, off, 2.0, 8, 7, 3)
    want = orc.cdcq_paths(1, None, th, y0, off, 2.0, 8, 7, 3)
    assert np.allclose(want[:300], math.exp(0.2), rtol=1e-12) and np.allclose(want[300:], 2 * math.exp(0.4), rtol=1e-12)
    assert np.all(rel_err(r["yt"], want, 1.0) <= 1e-6)


@pytest.mark.parametrize("n_steps", [1, 5])
def test_ragged_and_empty_sets(sl, orc, n_steps):
    P = W.near_affine_params(4, 7, seed=35)
    counts = [0, 1, 127, 128, 129, 0, 257]
    th = W.gbm_online_thetas(len(counts))
    y0 = np.linspace(0.8, 1.4, len(counts))
    off = W.offsets_from_counts(counts)
    r = _run(sl, 0, sl.make_net(_dev(P), 4, 7), th, y0, off, 1.0, n_steps, 7, 6, moments=True)
    _check(orc, r["yt"], orc.cdcq_paths(0, P, th, y0, off, 1.0, n_steps, 7, 6, d_in=4), off, 6, n_steps, 1.0)
    for s, c in enumerate(counts):
        seg = r["yt"][off[s]:off[s + 1]].astype(np.float64)
        assert r["mean"][s] == (pytest.approx(seg.mean(), rel=1e-12) if c else 0.0)


def test_batch_independence_and_graph(sl, orc):
    P = W.near_affine_params(5, 7, seed=36)
    net = sl.make_net(_dev(P), 5, 7)
    b = W.cir_batched(n_sets=300, lo_exp=1.0, hi_exp=3.0)
    off = b["offsets"]
    full = _run(sl, 0, net, b["theta"], b["Y0"], off, 4.0, 12, 7, 9)
    counts = np.diff(off)
    for s in (0, 137, int(np.argmax(counts))):
        only = np.zeros_like(counts)
        only[s] = counts[s]
        got = _run(sl, 0, net, b["theta"], b["Y0"], W.offsets_from_counts(only), 4.0, 12, 7, 9)["yt"]
        assert np.array_equal(got, full["yt"][off[s]:off[s + 1]]), s
    total = int(off[-1])
    th, y0, o = _dev(b["theta"]), _dev(b["Y0"]), _dev(off, torch.int64)
    yt = torch.empty(total, device="cuda")
    ws = torch.empty(sl.cdc_workspace_size(total, 300, 12), dtype=torch.uint8, device="cuda")
    run = lambda: sl.seven_league_cdc_simulate_batched(0, net, th, y0, o, 4.0, 12, 7, 9, out_YT=yt, ws=ws,
                                                       total_paths=total)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run()
    yt.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert sl.workspace_status(ws) == 0
    assert np.array_equal(yt.cpu().numpy(), full["yt"])
    idx = np.random.default_rng(3).integers(0, total, 1500)
    want = orc.cdcq_paths(0, P, b["theta"], b["Y0"], off, 4.0, 12, 7, 9, d_in=5, idx=idx)
    _check(orc, full["yt"][idx], want, off, 9, 12, 1.0, idx=idx)


def test_full_size_sampled(sl, orc):
    """16 parameter sets x 1e6 paths x 16 steps (T = 2, m = 7), sampled paths and the set means."""
    w = W.gbm_online()
    P = W.near_affine_params(4, 7, seed=0)
    off = w["offsets"]
    r = _run(sl, 0, sl.make_net(_dev(P), 4, 7), w["theta"], w["Y0"], off, w["T"], w["n_steps"], 7, w["seed"],
             moments=True)
    rng = np.random.default_rng(4)
    idx = np.unique(np.concatenate([rng.integers(0, int(off[-1]), 3000), off[1:] - 1, off[:-1]]))
    want = orc.cdcq_paths(0, P, w["theta"], w["Y0"], off, w["T"], w["n_steps"], 7, w["seed"], d_in=4, idx=idx)
    _check(orc, r["yt"][idx], want, off, w["seed"], w["n_steps"], 1.0, idx=idx)
    for s in range(16):
        seg = r["yt"][off[s]:off[s + 1]].astype(np.float64)
        assert r["mean"][s] == pytest.approx(seg.mean(), rel=1e-12)


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7, 8])
def test_every_m(sl, orc, m):
    th, y0 = [[0.1, 0.3], [0.05, 0.45]], [1.0, 2.0]
    off = W.offsets_from_counts([700, 1300])
    r = _run(sl, 1, None, th, y0, off, 1.0, 6, m, 5)
    _check(orc, r["yt"], orc.cdcq_paths(1, None, th, y0, off, 1.0, 6, m, 5), off, 5, 6, 1.0)


def test_more_than_2_31_paths(sl, orc):
    """One set of 2^31 + 129 paths, 2 steps, exact OU map: sampled paths including the last ones."""
    n = (1 << 31) + 129
    off = W.offsets_from_counts([n])
    th = [[0.5, 0.3, 1.0]]
    yt = torch.empty(n, dtype=torch.float32, device="cuda")
    mean = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = sl.seven_league_cdc_simulate_batched(2, None, _dev(th), _dev([1.5]), _dev(off, torch.int64), 1.0, 2, 7, 2,
                                              out_YT=yt, out_mean=mean)
    assert sl.workspace_status(ws) == 0
    idx = np.concatenate([np.arange(0, 64), np.arange((1 << 31) - 64, (1 << 31) + 64), np.arange(n - 64, n)])
    got = yt[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    _check(orc, got, orc.cdcq_paths(2, None, th, [1.5], off, 1.0, 2, 7, 2, idx=idx), off, 2, 2, 1.0, idx=idx)
    assert np.isfinite(mean.item())
    del yt


@pytest.mark.parametrize("model", [1, 2])
def test_exact_models_many_entries(sl, orc, model):
    """12,000 (set, step) entries with the exact maps (every CTA of the table kernel takes
    several rounds): the tables and sampled paths against the oracle."""
    n_sets, n_steps, m = 1000, 12, 7
    rng = np.random.default_rng(43 + model)
    counts = rng.integers(1, 4, n_sets)
    off = W.offsets_from_counts(counts)
    if model == 1:
        th = rng.uniform([0.0, 0.1], [0.2, 0.5], (n_sets, 2)).astype(np.float32)
        y0 = rng.uniform(0.8, 1.2, n_sets).astype(np.float32)
    else:
        th = rng.uniform([0.0, 0.1, 0.5], [1.0, 0.5, 2.0], (n_sets, 3)).astype(np.float32)
        y0 = rng.uniform(-0.5, 1.5, n_sets).astype(np.float32)
    r = _run(sl, model, None, th, y0, off, 3.0, n_steps, m, 5)
    sets = np.concatenate([np.arange(30), np.arange(n_sets - 30, n_sets)])
    zn, eta = orc.cdcq_tables(model, None, th, y0, 3.0, n_steps, m, sets=sets)
    _tables_vs_oracle(r["tab"][sets], zn, eta, m)
    idx = off[sets]
    _check(orc, r["yt"][idx], orc.cdcq_paths(model, None, th, y0, off, 3.0, n_steps, m, 5, idx=idx), off, 5, n_steps,
           1.0, idx=idx)


def test_many_sets(sl, orc):
    """2^20 parameter sets with 0 or 1 path each, 3 steps, a network."""
    n_sets = 1 << 20
    rng = np.random.default_rng(41)
    counts = rng.integers(0, 2, n_sets)
    off = W.offsets_from_counts(counts)
    th = rng.uniform([0.0, 0.1], [0.2, 0.5], (n_sets, 2)).astype(np.float32)
    y0 = rng.uniform(0.8, 1.2, n_sets).astype(np.float32)
    P = W.near_affine_params(4, 7, seed=42)
    r = _run(sl, 0, sl.make_net(_dev(P), 4, 7), th, y0, off, 1.0, 3, 7, 4, moments=True)
    sets = np.concatenate([np.nonzero(counts)[0][:40], np.nonzero(counts)[0][-40:]])
    idx = off[sets]
    _check(orc, r["yt"][idx], orc.cdcq_paths(0, P, th, y0, off, 1.0, 3, 7, 4, d_in=4, idx=idx), off, 4, 3, 1.0, idx=idx)
    assert np.array_equal(r["mean"][sets], r["yt"][idx].astype(np.float64)) and np.all(r["mean"][counts == 0] == 0)


def _double_crossing_nodes():
    """Nodes of G(xi) = 20 + (xi - 0.1)(xi - 0.135)(xi - 0.62) at the 4 Gauss-Hermite points:
    G exceeds 20 only on (0.1, 0.135), inside one 1/32 of the node interval [x_1, x_2]."""
    from numpy.polynomial import hermite_e
    x = hermite_e.hermegauss(4)[0]
    return (20.0 + (x - 0.1) * (x - 0.135) * (x - 0.62)).astype(np.float32)


def test_inverse_first_of_two_close_crossings(sl, orc):
    z = _double_crossing_nodes()
    ys = np.array([[20.0, 20.0 - 1e-5, 19.5, 20.5, float(z[1]), float(z[2]), float(z[0]) - 1.0, float(z[3]) + 3.0]])
    got = sl.cdcq_inverse(_dev(z[None, :]), _dev(ys, torch.float64)).cpu().numpy()[0]
    want = np.array([orc.cdcq_Ginv(z.astype(np.float64), y) for y in ys[0]])
    assert abs(want[0] - 0.1) < 1e-5 and abs(got[0] - 0.1) < 1e-5      # the first crossing, not 0.62
    assert np.allclose(got, want, rtol=0, atol=1e-9), (got, want)


@pytest.mark.parametrize("m", [4, 5, 6, 7, 8])
def test_inverse_of_wiggling_maps(sl, orc, m):
    """Random FP32 node sets that increase from first to last but wiggle between, 64 values of y
    each inside and around the range: the kernel's G^{-1} against the oracle's."""
    rng = np.random.default_rng(900 + m)
    zs, n_maps = [], 0
    while n_maps < 200:
        z = (np.cumsum(rng.uniform(-0.4, 1.0, size=m)) + rng.normal(size=m) * 0.3).astype(np.float32)
        if z[-1] > z[0]:
            zs.append(z)
            n_maps += 1
    zs = np.array(zs)
    ys = np.concatenate([rng.uniform(zs[:, :1] - 0.5, zs[:, -1:] + 0.5, size=(n_maps, 56)),
                         zs[:, :m].astype(np.float64), np.zeros((n_maps, 8 - m))], axis=1)
    ys = ys[:, :64]
    got = sl.cdcq_inverse(_dev(zs), _dev(ys, torch.float64)).cpu().numpy()
    want = np.array([[orc.cdcq_Ginv(zs[i].astype(np.float64), y) for y in ys[i]] for i in range(n_maps)])
    err = np.abs(got - want)
    print("max |xi - oracle|:", err.max())
    assert err.max() <= 1e-9


def test_inverse_degenerate_maps(sl, orc):
    zs = np.array([[0.7, 0.7, 0.7, 0.7, 0.7], [2.0, 1.0, 0.5, 0.2, 0.1], [0.0, 0.5, 1.0, 1.5, 2.0]], np.float32)
    ys = np.array([[3.0, 0.7], [0.5, 1.0], [0.75, 2.5]])
    got = sl.cdcq_inverse(_dev(zs), _dev(ys, torch.float64)).cpu().numpy()
    assert np.array_equal(got[0], [0.0, 0.0]) and np.all(np.isnan(got[1]))
    want = [orc.cdcq_Ginv(zs[2].astype(np.float64), y) for y in ys[2]]
    assert np.allclose(got[2], want, rtol=0, atol=1e-12)


def _passthrough_net(m, d_in, a, b5):
    """H_j(Y, .) = b5_j + a_j max(Y, 0): unit 0 of every hidden layer carries Y, the rest are 0."""
    P = np.zeros(sum([50 * d_in + 50] + [50 * 50 + 50] * 3 + [m * 50 + m]), np.float32)
    off = 0
    P[off + 0] = 1.0                       # W1[0][0]: the Y feature
    off += 50 * d_in + 50
    for _ in range(3):
        P[off + 0] = 1.0                   # W_l[0][0]
        off += 50 * 50 + 50
    for j in range(m):
        P[off + j * 50] = a[j]             # W5[j][0]
    P[off + m * 50:off + m * 50 + m] = b5
    return P


def test_tables_take_the_first_of_two_close_crossings(sl, orc):
    """A network with H_j(Y) = b5_j + a_j Y (Y > 0): the marginal nodes of every t_i > 0 are the
    double-crossing nodes z, and the conditional point C[3][1] = H_1(z_3) = 20, so at step 1
    eta[3][1] = G^{-1}(20) must be the first crossing (0.1), as in the oracle."""
    m, d_in, y0 = 4, 3, 1.0
    z = _double_crossing_nodes().astype(np.float64)
    a = np.zeros(m)
    a[1] = (20.0 - z[1]) / (z[3] - y0)
    b5 = z - a * y0
    P = _passthrough_net(m, d_in, a.astype(np.float32), b5.astype(np.float32))
    th, y0s, off = [[0.0]], [y0], W.offsets_from_counts([256])
    r = _run(sl, 0, sl.make_net(_dev(P), d_in, m), th, y0s, off, 1.0, 2, m, 3)
    zn, eta = orc.cdcq_tables(0, P, th, y0s, 1.0, 2, m, d_in=d_in)
    ge = r["tab"][0, 1, 24:88].reshape(8, 8)[:m, :m].astype(np.float64)
    assert abs(eta[0, 1, 3, 1] - 0.1) < 1e-3 and abs(ge[3, 1] - 0.1) < 1e-3
    assert np.abs(ge - eta[0, 1]).max() <= 1e-3          # y moves by an FP32 rounding, xi by ~1/G'
