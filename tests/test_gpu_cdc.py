"""GPU parity of the 7L-CDC sampler (network evaluations at the marginal collocation
points, interpolation in Y per path) against the FP64 oracle, through the C ABI.

Tolerance: TOL * kappa on |a - b| / (|b| + s) per path, gated like the FP32 7L sampler (paths
whose normals stay within |X| <= 4, plus the 99.99th percentile over all paths).  The GPU side
is FP32 throughout (table entries, the interpolation in Y and g_m) against FP64 on the same
normals.  The interpolation in Y sums terms L_k(Y) C[k][j] that can be far larger than their
sum: through the quantile nodes of a wide lognormal marginal (sigma sqrt(t) ~ 0.7, nodes spread
over a factor ~170) sum_k |L_k(Y)| |C[k][j]| / |yhat_j| reaches ~2500 inside the nodes' hull,
and FP32 rounding of the table entries is magnified by that factor in any evaluation order.
kappa is that condition number, max over the path's steps of
sum_k |L_k(Y_i)| max_j |C[k][j]| / (max_j |yhat_j| + s) inside the nodes' hull and of
max_j (|C[a][j]| + |Y_i - z_a| (|C[a][j]| + |C[b][j]|) / |z_b - z_a|) / (max_j |yhat_j| + s)
on the continuation line through nodes a, b beyond it, computed below with numpy from the
oracle's own FP64 path and tables (1 for a well-conditioned path).

* Exact GBM and OU maps (where the chain equals the 7L chain) against the oracle, and against
  the GPU's own FP32 7L sampler on the same normals; m = 2..8.
* Networks (ReLU, Softplus, a separate marginal network): the tables the call leaves in its
  workspace (marginal nodes, their barycentric weights, conditional points) against the
  oracle's, and the paths.  The networks are workloads.near_affine_params (outputs shaped like
  collocation points, plus a perturbation that switches ReLU units): an untrained Xavier
  network's marginal points are unordered or nearly coincide, and the interpolation in Y
  through them diverges (the status word then reports non-finite paths).
* Degenerate laws (sigma = 0: every marginal collapses to a point), ragged and empty sets,
  one step, batch independence (bit-exact), CUDA graph replay, FP64 set moments, the full
  16 x 1e6 x 16 workload on sampled paths, 2^31 + 129 paths in one set, 2^20 sets.
"""
import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W
from tests.helpers import flat_sets, gate, max_abs_normals, rel_err

pytestmark = pytest.mark.gpu
# per step: FP32 rounding of the table entries (network evaluations of condition ~4: a few
# 1e-7 relative) and of the two interpolations, magnified by kappa, accumulated over up to
# 16 steps: ~2e-5 at most; measured max 1.1e-5 (16 steps, full size)
TOL = 3e-5


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _run(sl, model, net, theta, Y0, offsets, T, n_steps, m, seed, marg=None, grid=False, moments=False):
    total = int(offsets[-1])
    n_sets = len(offsets) - 1
    yt = torch.full((max(total, 1),), float("nan"), dtype=torch.float32, device="cuda")
    gr = torch.empty((n_steps + 1, total), dtype=torch.float32, device="cuda") if grid else None
    mean = torch.full((n_sets,), float("nan"), dtype=torch.float64, device="cuda") if moments else None
    var = torch.empty_like(mean) if moments else None
    ws = sl.seven_league_cdc_simulate_batched(model, net, _dev(theta), _dev(Y0), _dev(offsets, torch.int64), T,
                                              n_steps, m, seed, marg_net=marg, space=sl.CDC_Y, out_YT=yt,
                                              out_grid=gr, out_mean=mean, out_var=var)
    assert sl.workspace_status(ws) == 0
    tab = sl.cdc_tables(ws, n_sets, n_steps).cpu().numpy()
    out = dict(yt=yt.cpu().numpy()[:total], tab=tab)
    if grid:
        out["grid"] = gr.cpu().numpy()
    if moments:
        out["mean"], out["var"] = mean.cpu().numpy(), var.cpu().numpy()
    return out


def _kappa(z, C, grid, sets, scale):
    """Per path: max over steps of the condition number of the interpolation in Y (see the
    module docstring); z [n_sets, n_steps, m], C [n_sets, n_steps, m, m], grid [n, n_steps+1]."""
    n_steps, m = z.shape[1], z.shape[2]
    kap = np.ones(grid.shape[0])
    for i in range(1, n_steps):
        zi, Ci, Y = z[sets, i], C[sets, i], grid[:, i]
        live = np.any(zi != zi[:, :1], axis=1)
        if not live.any():
            continue
        zi, Ci, Y = zi[live], Ci[live], Y[live]
        L = np.ones((zi.shape[0], m))
        for k in range(m):
            for l in range(m):
                if l != k:
                    L[:, k] *= (Y - zi[:, l]) / (zi[:, k] - zi[:, l])
        yh = np.einsum("nk,nkj->nj", L, Ci)
        kk = np.einsum("nk,nk->n", np.abs(L), np.abs(Ci).max(axis=2)) / (np.abs(yh).max(axis=1) + scale)
        order = np.argsort(zi, axis=1, kind="stable")
        rows = np.arange(len(Y))
        for a_col, b_col, outside in ((0, 1, Y < zi.min(axis=1)), (-1, -2, Y > zi.max(axis=1))):
            if not outside.any():
                continue
            a, b = order[:, a_col], order[:, b_col]
            za, zb, Ca, Cb = zi[rows, a], zi[rows, b], Ci[rows, a], Ci[rows, b]
            line = Ca + ((Y - za) / (zb - za))[:, None] * (Cb - Ca)
            ko = (np.abs(Ca) + (np.abs(Y - za) / np.abs(zb - za))[:, None] * (np.abs(Ca) + np.abs(Cb))).max(axis=1)
            kk = np.where(outside, ko / (np.abs(line).max(axis=1) + scale), kk)
        kap[live] = np.maximum(kap[live], kk)
    return kap


def _oracle(orc, model, P, theta, Y0, offsets, T, n_steps, m, seed, scale, Pm=None, idx=None, d_in=3, act=0):
    """The oracle's Y_T of the selected paths and their kappa."""
    yt, grid = orc.cdc_paths(model, P, theta, Y0, offsets, T, n_steps, m, seed, Pm=Pm, idx=idx, d_in=d_in,
                             act=act, grid=True)
    idx = np.arange(len(yt)) if idx is None else idx
    sets, _ = flat_sets(offsets, idx)
    used = np.unique(sets)
    z, C = orc.cdc_tables(model, P, theta, Y0, T, n_steps, m, Pm=Pm, d_in=d_in, act=act, sets=used)
    return yt, _kappa(z, C, grid, np.searchsorted(used, sets), scale)


def _check(orc, got, want, offsets, seed, n_steps, scale, idx=None, tol=TOL):
    want, kappa = want
    idx = np.arange(len(want)) if idx is None else idx
    s, q = flat_sets(offsets, idx)
    err = rel_err(got, want, scale) / kappa
    ok, *info = gate(err, max_abs_normals(orc, seed, 0, s, q, n_steps), tol)
    print("per-path error / kappa (max |X|<=4, p99.99, max):", info, "kappa max %.3g" % kappa.max())
    assert ok, info


@pytest.mark.parametrize("model,theta,Y0,m", [
    (1, [[0.1, 0.3], [0.15, 0.5], [0.0, 0.1]], [1.0, 0.7, 3.0], 7),
    (2, [[0.5, 0.3, 1.0], [1.0, 0.45, 0.6]], [1.5, -0.5], 5),
])
def test_exact_models_vs_oracle_and_7l(sl, orc, model, theta, Y0, m):
    off = W.offsets_from_counts([3000 + 1111 * s for s in range(len(Y0))])
    r = _run(sl, model, None, theta, Y0, off, 2.0, 16, m, 21)
    want = _oracle(orc, model, None, theta, Y0, off, 2.0, 16, m, 21, 1.0)
    _check(orc, r["yt"], want, off, 21, 16, 1.0)
    yt7 = torch.empty(int(off[-1]), device="cuda")
    ws = sl.seven_league_simulate_batched(model, None, _dev(theta), _dev(Y0), _dev(off, torch.int64), 2.0, 16, m,
                                          21, out_YT=yt7)
    assert sl.workspace_status(ws) == 0
    _check(orc, r["yt"], (yt7.cpu().numpy(), want[1]), off, 21, 16, 1.0)


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7, 8])
def test_every_m(sl, orc, m):
    th, y0 = [[0.1, 0.3], [0.05, 0.45]], [1.0, 2.0]
    off = W.offsets_from_counts([700, 1300])
    r = _run(sl, 1, None, th, y0, off, 1.0, 6, m, 5)
    _check(orc, r["yt"], _oracle(orc, 1, None, th, y0, off, 1.0, 6, m, 5, 1.0), off, 5, 6, 1.0)


def _gh_monomials(m):
    """[j][a]: monomial coefficients of b_j prod_{l!=j} (X - x_l) from numpy's Gauss-Hermite points."""
    from numpy.polynomial import hermite_e, polynomial as Pn
    x = hermite_e.hermegauss(m)[0]
    out = np.zeros((m, m))
    for j in range(m):
        c = np.array([1.0])
        for l in range(m):
            if l != j:
                c = Pn.polymul(c, [-x[l], 1.0])
        out[j] = c / np.prod([x[j] - x[l] for l in range(m) if l != j])
    return out


def _tables_vs_oracle(tab, z, C, m, tol):
    n_sets, n_steps = z.shape[:2]
    gz = tab[:, :, :m].astype(np.float64)
    gw = tab[:, :, 8:8 + m].astype(np.float64)
    gC = tab[:, :, 16:80].reshape(n_sets, n_steps, 8, 8)[:, :, :m, :m].astype(np.float64)
    scale = np.abs(z).max()
    assert np.all(tab[:, :, m:8] == 0) and np.all(tab[:, :, 8 + m:16] == 0)
    assert np.abs(gz - z).max() <= tol * scale
    assert np.abs(gC - C).max() <= tol * np.abs(C).max()
    assert np.all(gw[:, 0] == 0)                                    # step 0: the point mass at Y0
    # weights are 1/prod(z_k - z_l) of the kernel's own FP32 nodes (FP64 products, one rounding)
    zz = tab[:, 1:, :m].astype(np.float64)
    want_w = 1.0 / np.prod(zz[..., :, None] - zz[..., None, :] + np.eye(m), axis=-1)
    assert np.allclose(gw[:, 1:], want_w, rtol=2 ** -23, atol=0)
    # continuation lines: outermost nodes, their rows, slopes of the two outermost nodes
    t = tab[:, 1:].astype(np.float64)
    zc = t[..., :m]
    Cc = t[..., 16:80].reshape(n_sets, n_steps - 1, 8, 8)[..., :m, :m]
    order = np.argsort(zc, axis=-1, kind="stable")
    take = lambda A, o: np.take_along_axis(A, o[..., None, None].repeat(m, -1), axis=-2)[..., 0, :]
    for (a, b, zcol, ccol, scol) in ((0, 1, 112, 96, 80), (m - 1, m - 2, 113, 104, 88)):
        ia, ib = order[..., a], order[..., b]
        za = np.take_along_axis(zc, ia[..., None], -1)[..., 0]
        zb = np.take_along_axis(zc, ib[..., None], -1)[..., 0]
        assert np.array_equal(t[..., zcol], za)
        assert np.array_equal(t[..., ccol:ccol + m], take(Cc, ia))
        slope = (take(Cc, ib) - take(Cc, ia)) / (zb - za)[..., None]
        assert np.allclose(t[..., scol:scol + m], slope, rtol=2 ** -23, atol=0)
    assert np.all(tab[:, :, 114:120] == 0)
    # monomial rows of g_m: coefficient a of sum_j y_j b_j Q_j(X), Q_j = prod_{l!=j} (X - x_l), for
    # y = row k of C times w_k (A), row 0 (D), the outer rows and slopes (B, Sm); FP64 from the
    # kernel's own FP32 entries, one rounding (the tolerance scales with the summands' size)
    bq = _gh_monomials(m)                                              # [j][a]
    t0 = tab.astype(np.float64)
    Call = t0[..., 16:80].reshape(n_sets, n_steps, 8, 8)[..., :m, :m]
    wall = t0[..., 8:8 + m]
    def near(got, rows, scale_rows):
        want = rows @ bq
        size = np.abs(scale_rows) @ np.abs(bq)
        assert np.all(np.abs(got - want) <= 2 ** -21 * size + 1e-30), np.abs(got - want).max()
    A = t0[..., 128:192].reshape(n_sets, n_steps, 8, 8)[..., :m, :m]
    near(A, wall[..., :, None] * Call, wall[..., :, None] * Call)
    near(t0[..., 120:120 + m], Call[..., 0, :], Call[..., 0, :])
    for zcol, ccol, scol, bcol, smcol in ((112, 96, 80, 192, 200), (113, 104, 88, 208, 216)):
        near(t0[..., bcol:bcol + m], t0[..., ccol:ccol + m], t0[..., ccol:ccol + m])
        live = wall[..., 0] != 0
        sm = t0[..., smcol:smcol + m]
        want = t0[..., scol:scol + m] @ bq
        size = (np.abs(t0[..., scol:scol + m]) @ np.abs(bq))
        assert np.all(np.abs(sm - want)[live] <= (2 ** -20 * size + 1e-30)[live])
    assert np.all(tab[:, :, 120 + m:128] == 0) and np.all(tab[:, 0, 128:192] == 0)


@pytest.mark.parametrize("act", [0, 1])
def test_network_tables_and_paths(sl, orc, act):
    d_in, m, n_steps = 4, 7, 8
    P = W.near_affine_params(d_in, m, seed=11)
    net = sl.make_net(_dev(P), d_in, m, act=act)
    th = W.gbm_online_thetas(3)
    y0 = [1.0, 0.8, 1.3]
    off = W.offsets_from_counts([2500, 1, 3333])
    r = _run(sl, 0, net, th, y0, off, 2.0, n_steps, m, 8)
    z, C = orc.cdc_tables(0, P, th, y0, 2.0, n_steps, m, d_in=d_in, act=act)
    _tables_vs_oracle(r["tab"], z, C, m, 1e-5)
    want = _oracle(orc, 0, P, th, y0, off, 2.0, n_steps, m, 8, 1.0, d_in=d_in, act=act)
    _check(orc, r["yt"], want, off, 8, n_steps, 1.0)


def test_separate_marginal_network(sl, orc):
    d_in, m, n_steps = 5, 5, 6
    P, Pm = W.near_affine_params(d_in, m, seed=12), W.near_affine_params(d_in, m, b=0.4, seed=13)
    net = sl.make_net(_dev(P), d_in, m)
    mnet = sl.make_net(_dev(Pm), d_in, m, act=1)                      # Softplus marginal network
    th, y0 = [[0.5, 0.3, 1.0], [0.2, 0.4, 1.5]], [1.5, 0.0]
    off = W.offsets_from_counts([1500, 900])
    r = _run(sl, 0, net, th, y0, off, 1.5, n_steps, m, 4, marg=mnet)
    # the oracle takes one activation for both networks: check the nodes against the
    # Softplus marginal network directly, and the rest against the tables built from them
    f = np.array([[y0[s], 0.25 * i] + th[s] for s in range(2) for i in range(1, n_steps)])
    zm = orc.mlp_forward(Pm, f, d_in, m, act=1).reshape(2, n_steps - 1, m)
    assert np.abs(r["tab"][:, 1:, :m] - zm).max() <= 1e-5 * np.abs(zm).max()
    gz = r["tab"][:, :, :m].astype(np.float64)
    C = orc.mlp_forward(P, np.concatenate([gz.reshape(-1, 1), np.repeat(
        np.array([[0.25] + th[s] for s in range(2)]), n_steps * m, 0)], 1), d_in, m).reshape(2, n_steps, m, m)
    gC = r["tab"][:, :, 16:80].reshape(2, n_steps, 8, 8)[:, :, :m, :m]
    assert np.abs(gC - C).max() <= 1e-5 * np.abs(C).max()


def test_degenerate_law(sl, orc):
    """sigma = 0: every marginal is a point, every table row takes the degenerate branch and
    the chain is the deterministic growth Y0 exp(mu T)."""
    th, y0 = [[0.1, 0.0], [0.2, 0.0]], [1.0, 2.0]
    off = W.offsets_from_counts([300, 200])
    r = _run(sl, 1, None, th, y0, off, 2.0, 8, 7, 3)
    assert np.all(r["tab"][:, :, 8:16] == 0)
    want = orc.cdc_paths(1, None, th, y0, off, 2.0, 8, 7, 3)
    assert np.allclose(want[:300], np.exp(0.2), rtol=1e-12) and np.allclose(want[300:], 2 * np.exp(0.4), rtol=1e-12)
    assert np.all(rel_err(r["yt"], want, 1.0) <= 1e-6)


@pytest.mark.parametrize("n_steps", [1, 5])
def test_ragged_and_empty_sets(sl, orc, n_steps):
    P = W.near_affine_params(4, 7, seed=14)
    net = sl.make_net(_dev(P), 4, 7)
    counts = [0, 1, 127, 128, 129, 0, 257]
    th = W.gbm_online_thetas(len(counts))
    y0 = np.linspace(0.8, 1.4, len(counts))
    off = W.offsets_from_counts(counts)
    r = _run(sl, 0, net, th, y0, off, 1.0, n_steps, 7, 6, moments=True)
    want = _oracle(orc, 0, P, th, y0, off, 1.0, n_steps, 7, 6, 1.0, d_in=4)
    _check(orc, r["yt"], want, off, 6, n_steps, 1.0)
    for s, c in enumerate(counts):
        seg = r["yt"][off[s]:off[s + 1]].astype(np.float64)
        assert r["mean"][s] == (pytest.approx(seg.mean(), rel=1e-12) if c else 0.0)
    if n_steps == 1:     # one step: the 7L-CDC chain is the 7L chain (network at Y0)
        yt7 = torch.empty(int(off[-1]), device="cuda")
        ws = sl.seven_league_simulate_batched(0, net, _dev(th), _dev(y0), _dev(off, torch.int64), 1.0, 1, 7, 6,
                                              out_YT=yt7)
        assert sl.workspace_status(ws) == 0
        assert np.all(rel_err(r["yt"], yt7.cpu().numpy(), 1.0) <= 1e-5)


def test_no_paths(sl, orc):
    off = W.offsets_from_counts([0, 0])
    r = _run(sl, 1, None, [[0.1, 0.3], [0.1, 0.3]], [1.0, 1.0], off, 1.0, 4, 5, 1, moments=True)
    assert r["yt"].size == 0 and np.all(r["mean"] == 0)


def test_batch_independence_graph_and_grid(sl, orc):
    P = W.near_affine_params(5, 7, seed=15)
    net = sl.make_net(_dev(P), 5, 7)
    b = W.cir_batched(n_sets=300, lo_exp=1.0, hi_exp=3.0)
    off = b["offsets"]
    full = _run(sl, 0, net, b["theta"], b["Y0"], off, 4.0, 12, 7, 9, grid=True)
    assert np.array_equal(full["grid"][-1], full["yt"]) and np.all(full["grid"][0] == np.repeat(b["Y0"], np.diff(off)))
    counts = np.diff(off)
    for s in (0, 137, int(np.argmax(counts))):
        only = np.zeros_like(counts)
        only[s] = counts[s]
        got = _run(sl, 0, net, b["theta"], b["Y0"], W.offsets_from_counts(only), 4.0, 12, 7, 9)["yt"]
        assert np.array_equal(got, full["yt"][off[s]:off[s + 1]]), s
    total = int(off[-1])
    th, y0, o = _dev(b["theta"]), _dev(b["Y0"]), _dev(off, torch.int64)
    yt = torch.empty(total, device="cuda")
    mean = torch.empty(300, dtype=torch.float64, device="cuda")
    ws = torch.empty(sl.cdc_workspace_size(total, 300, 12), dtype=torch.uint8, device="cuda")
    run = lambda: sl.seven_league_cdc_simulate_batched(0, net, th, y0, o, 4.0, 12, 7, 9, space=sl.CDC_Y, out_YT=yt,
                                                       out_mean=mean, ws=ws, total_paths=total)
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
    idx = np.random.default_rng(1).integers(0, total, 1500)
    # the near-affine network spreads the state over ~1 whatever the CIR parameters: scale 1
    want = _oracle(orc, 0, P, b["theta"], b["Y0"], off, 4.0, 12, 7, 9, 1.0, d_in=5, idx=idx)
    _check(orc, full["yt"][idx], want, off, 9, 12, 1.0, idx=idx)


def test_full_size_sampled(sl, orc):
    """16 parameter sets x 1e6 paths x 16 steps (T = 2, m = 7), sampled paths and the set means."""
    w = W.gbm_online()
    P = W.near_affine_params(4, 7, seed=0)
    net = sl.make_net(_dev(P), 4, 7)
    off = w["offsets"]
    r = _run(sl, 0, net, w["theta"], w["Y0"], off, w["T"], w["n_steps"], 7, w["seed"], moments=True)
    rng = np.random.default_rng(2)
    idx = np.unique(np.concatenate([rng.integers(0, int(off[-1]), 3000), off[1:] - 1, off[:-1]]))
    want = _oracle(orc, 0, P, w["theta"], w["Y0"], off, w["T"], w["n_steps"], 7, w["seed"], 1.0, d_in=4, idx=idx)
    _check(orc, r["yt"][idx], want, off, w["seed"], w["n_steps"], 1.0, idx=idx)
    for s in range(16):
        seg = r["yt"][off[s]:off[s + 1]].astype(np.float64)
        assert r["mean"][s] == pytest.approx(seg.mean(), rel=1e-12)


def test_more_than_2_31_paths(sl, orc):
    """One set of 2^31 + 129 paths (flat and in-set indices past int32), 2 steps, exact GBM map:
    sampled paths including the last ones against the oracle; the set mean is finite."""
    n = (1 << 31) + 129
    off = W.offsets_from_counts([n])
    th = [[0.1, 0.3]]
    yt = torch.empty(n, dtype=torch.float32, device="cuda")
    mean = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = sl.seven_league_cdc_simulate_batched(1, None, _dev(th), _dev([1.0]), _dev(off, torch.int64), 1.0, 2, 7, 2,
                                              space=sl.CDC_Y, out_YT=yt, out_mean=mean)
    assert sl.workspace_status(ws) == 0
    idx = np.concatenate([np.arange(0, 64), np.arange((1 << 31) - 64, (1 << 31) + 64), np.arange(n - 64, n)])
    got = yt[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    want = _oracle(orc, 1, None, th, [1.0], off, 1.0, 2, 7, 2, 1.0, idx=idx)
    _check(orc, got, want, off, 2, 2, 1.0, idx=idx)
    assert np.isfinite(mean.item())
    del yt


def test_many_sets(sl, orc):
    """2^20 parameter sets with 0 or 1 path each, 3 steps, a network: 3 * 2^20 table entries."""
    n_sets = 1 << 20
    rng = np.random.default_rng(21)
    counts = rng.integers(0, 2, n_sets)
    off = W.offsets_from_counts(counts)
    th = rng.uniform([0.0, 0.1], [0.2, 0.5], (n_sets, 2)).astype(np.float32)
    y0 = rng.uniform(0.8, 1.2, n_sets).astype(np.float32)
    P = W.near_affine_params(4, 7, seed=22)
    net = sl.make_net(_dev(P), 4, 7)
    r = _run(sl, 0, net, th, y0, off, 1.0, 3, 7, 4, moments=True)
    sets = np.concatenate([np.nonzero(counts)[0][:40], np.nonzero(counts)[0][-40:]])
    idx = off[sets]
    want = _oracle(orc, 0, P, th, y0, off, 1.0, 3, 7, 4, 1.0, idx=idx, d_in=4)
    _check(orc, r["yt"][idx], want, off, 4, 3, 1.0, idx=idx)
    assert np.array_equal(r["mean"][sets], r["yt"][idx].astype(np.float64)) and np.all(r["mean"][counts == 0] == 0)
