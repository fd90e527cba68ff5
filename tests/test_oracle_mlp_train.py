"""Pins of the oracle's network H (Eq. 6.3/6.4), its gradients and Adam.

* Forward pass vs torch.nn.Linear/ReLU/Softplus layers in FP64 (an independent
  library implementation of the same fully connected network).
* Parameter gradient of the MSE loss vs central finite differences and vs
  torch.autograd.
* Input vector-Jacobian product vs central finite differences.
* Adam steps vs torch.optim.Adam on the same network and minibatches, and the
  closed form of Adam's first step (|update| = lr for |g| >> eps).
"""
import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W


def _torch_net(P, d_in, m, act):
    layers = []
    for li, (Wt, b) in enumerate(W.split_params(np.asarray(P, np.float64), d_in, m)):
        lin = torch.nn.Linear(Wt.shape[1], Wt.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(Wt.copy()))
            lin.bias.copy_(torch.from_numpy(b.copy()))
        layers.append(lin)
        if li < W.N_HIDDEN:
            layers.append(torch.nn.ReLU() if act == 0 else torch.nn.Softplus())
    return torch.nn.Sequential(*layers)


def _params(d_in, m, seed, bias_scale=0.1):
    P = W.xavier_params(d_in, m, seed=seed).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    # give the biases non-zero values so that their wiring is exercised
    o = 0
    for (fo, fi) in W.layer_shapes(d_in, m):
        o += fo * fi
        P[o:o + fo] = rng.uniform(-bias_scale, bias_scale, fo)
        o += fo
    return P


@pytest.mark.parametrize("act", [0, 1])
@pytest.mark.parametrize("d_in,m", [(3, 5), (4, 7), (5, 7)])
def test_forward_vs_torch(orc, act, d_in, m):
    P = _params(d_in, m, seed=d_in * 10 + m)
    rng = np.random.default_rng(1)
    f = rng.uniform(-1, 2, size=(64, d_in))
    got = orc.mlp_forward(P, f, d_in, m, act=act)
    net = _torch_net(P, d_in, m, act)
    want = net(torch.from_numpy(f)).detach().numpy()
    assert np.allclose(got, want, rtol=1e-12, atol=1e-13)
    assert orc.n_params(d_in, m) == W.n_params(d_in, m) == sum(p.numel() for p in net.parameters())


@pytest.mark.parametrize("act", [0, 1])
def test_param_gradient(orc, act):
    d_in, m = 4, 7
    P = _params(d_in, m, seed=3)
    rng = np.random.default_rng(2)
    f = rng.uniform(-1, 2, size=(16, d_in))
    y = rng.standard_normal((16, m))
    loss, g = orc.mse_grad(P, f, y, d_in, m, act=act)
    # torch autograd
    net = _torch_net(P, d_in, m, act)
    lt = torch.mean((net(torch.from_numpy(f)) - torch.from_numpy(y)) ** 2)
    lt.backward()
    gt = np.concatenate([p.grad.numpy().ravel() for p in net.parameters()])
    assert loss == pytest.approx(lt.item(), rel=1e-13)
    assert np.allclose(g, gt, rtol=1e-10, atol=1e-13)
    # central differences on a sample of coordinates (one in every layer)
    h = 1e-6
    idx = np.unique(np.concatenate([rng.integers(0, P.size, 40), [0, 199, 200, 2750, P.size - 1]]))
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (orc.mse_grad(Pp, f, y, d_in, m, act=act)[0] - orc.mse_grad(Pm, f, y, d_in, m, act=act)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_row_selection(orc):
    d_in, m = 3, 5
    P = _params(d_in, m, seed=4)
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, size=(20, d_in))
    y = rng.standard_normal((20, m))
    rows = np.array([3, 7, 7, 19], dtype=np.int32)
    l1, g1 = orc.mse_grad(P, f, y, d_in, m, rows=rows)
    l2, g2 = orc.mse_grad(P, f[rows], y[rows], d_in, m)
    assert l1 == l2 and np.array_equal(g1, g2)


@pytest.mark.parametrize("act", [0, 1])
def test_input_vjp(orc, act):
    d_in, m = 5, 7
    P = _params(d_in, m, seed=5)
    rng = np.random.default_rng(4)
    f = rng.uniform(-0.5, 1.5, size=(8, d_in))
    c = rng.standard_normal((8, m))
    g = orc.mlp_vjp_input(P, f, c, d_in, m, act=act)
    h = 1e-6
    for k in range(d_in):
        fp, fm = f.copy(), f.copy()
        fp[:, k] += h
        fm[:, k] -= h
        fd = ((orc.mlp_forward(P, fp, d_in, m, act=act) - orc.mlp_forward(P, fm, d_in, m, act=act)) * c).sum(1) / (2 * h)
        assert np.allclose(g[:, k], fd, rtol=1e-5, atol=1e-8)


def test_adam_vs_torch(orc):
    d_in, m, batch, nb = 4, 7, 32, 6
    P = _params(d_in, m, seed=6)
    rng = np.random.default_rng(5)
    f = rng.uniform(0, 1, size=(200, d_in))
    y = rng.standard_normal((200, m))
    rows = W.minibatch_rows(200, batch, nb, seed=9)
    P2, am, av, losses = orc.train_adam(P, np.zeros_like(P), np.zeros_like(P), 0, f, y, rows, batch,
                                        d_in, m, lr=1e-3)
    net = _torch_net(P, d_in, m, 0)
    opt = torch.optim.Adam(net.parameters(), lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    tl = []
    for b in range(nb):
        opt.zero_grad()
        r = torch.from_numpy(rows[b].astype(np.int64))
        loss = torch.mean((net(torch.from_numpy(f)[r]) - torch.from_numpy(y)[r]) ** 2)
        loss.backward()
        tl.append(loss.item())
        opt.step()
    Pt = np.concatenate([p.detach().numpy().ravel() for p in net.parameters()])
    assert np.allclose(losses, tl, rtol=1e-12)
    assert np.allclose(P2, Pt, rtol=1e-9, atol=1e-12)


def test_adam_first_step_closed_form(orc):
    d_in, m, batch = 3, 5, 16
    P = _params(d_in, m, seed=7)
    rng = np.random.default_rng(6)
    f = rng.uniform(0, 1, size=(batch, d_in))
    y = rng.standard_normal((batch, m))
    rows = np.arange(batch, dtype=np.int32)[None, :]
    _, g = orc.mse_grad(P, f, y, d_in, m)
    P1, _, _, _ = orc.train_adam(P, np.zeros_like(P), np.zeros_like(P), 0, f, y, rows, batch, d_in, m,
                                 lr=1e-3)
    # first bias-corrected step: m_hat = g, v_hat = g^2, update = lr * g / (|g| + eps)
    want = P - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.allclose(P1, want, rtol=0, atol=1e-15)
    big = np.abs(g) > 1e-4
    assert np.allclose(np.abs(P1 - P)[big], 1e-3, rtol=1e-4)
