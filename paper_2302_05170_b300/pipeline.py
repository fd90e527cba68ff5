"""Offline stage of the 7L scheme (Algorithm I, step 1), end to end on the GPU.

Label rows (theta, Y_i, dt) -> em_collocation_labels (fine-step Euler-Maruyama
and empirical quantiles at Phi(x_j)) -> Adam training of the network on
(Y_i, dt, theta) -> labels, in the library's kernels.  Adam with batch 1024
and learning rate 1e-3 are the experiments section's settings; the rate then
decays geometrically to lr_end over the run (piecewise constant, n_chunks
pieces), because at a fixed 1e-3 the Adam noise keeps the network's per-step
error, and so the sampler's strong error, from settling.

Optional, both off by default:
* normalize: the network is trained on features and labels shifted and scaled
  to mean 0 and variance 1 per column, and the two affine maps are then folded
  into the first and the last layer, so the returned network takes and gives
  the raw values (the paper leaves input scaling open);
* bf16_steps: after the FP32 training, that many Adam steps train the network
  whose weights and biases are rounded to BF16 -- the one the tensor-core
  sampler evaluates -- with the FP32 parameters as the master copy; the
  result is then rounded to BF16 values, so the FP32 and the tensor-core
  forms run the same trained network.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W


def fold_normalization(P, d_in, m, f_shift, f_scale, y_shift, y_scale):
    """The network that maps raw features to raw labels, from one trained on
    (f - f_shift) / f_scale -> (y - y_shift) / y_scale: W1 / f_scale per input column and
    b1 - W1 (f_shift / f_scale) in the first layer, y_scale W5 and y_scale b5 + y_shift in
    the last.  P: flat FP32 tensor (layout of workloads.layer_shapes); returns a new one."""
    import torch
    P = P.clone()
    shapes = W.layer_shapes(d_in, m)
    o = 0
    offs = []
    for fo, fi in shapes:
        offs.append((o, o + fo * fi, fo, fi))
        o += fo * fi + fo
    w1o, b1o, fo1, fi1 = offs[0]
    W1 = P[w1o:w1o + fo1 * fi1].view(fo1, fi1).double()
    fsh, fsc = torch.as_tensor(f_shift, dtype=torch.float64, device=P.device), torch.as_tensor(
        f_scale, dtype=torch.float64, device=P.device)
    P[b1o:b1o + fo1] = (P[b1o:b1o + fo1].double() - W1 @ (fsh / fsc)).float()
    P[w1o:w1o + fo1 * fi1] = (W1 / fsc[None, :]).reshape(-1).float()
    w5o, b5o, fo5, fi5 = offs[-1]
    ysh, ysc = torch.as_tensor(y_shift, dtype=torch.float64, device=P.device), torch.as_tensor(
        y_scale, dtype=torch.float64, device=P.device)
    P[w5o:w5o + fo5 * fi5] = (P[w5o:w5o + fo5 * fi5].view(fo5, fi5).double() * ysc[:, None]).reshape(-1).float()
    P[b5o:b5o + fo5] = (P[b5o:b5o + fo5].double() * ysc + ysh).float()
    return P


def _adam_chunks(sl, P, d_in, m, feats, labels, n_steps, batch, lr0, lr_end, n_chunks, act, prec, shuffle_seed, ws):
    import torch
    am, av = torch.zeros_like(P), torch.zeros_like(P)
    n_rows = feats.shape[0]
    per = max(1, n_steps // n_chunks)
    losses, t0 = [], 0
    for c in range(n_chunks):
        lr = lr0 * (lr_end / lr0) ** (c / max(1, n_chunks - 1))
        rows = torch.as_tensor(W.minibatch_rows(n_rows, batch, per, seed=shuffle_seed + c), device=P.device)
        losses.append(sl.train(P, d_in, m, am, av, t0, feats, labels, rows, batch, lr=float(lr), act=act, ws=ws,
                               prec=prec))
        t0 += per
    return losses


def train_network(sde, theta, Yi, dt, m, n_paths=100_000, n_fine=100, label_seed=7, n_steps=40_000,
                  batch=1024, lr0=1e-3, lr_end=1e-5, n_chunks=20, act=0, init_seed=0, shuffle_seed=3,
                  normalize=False, bf16_steps=0, bf16_lr=(1e-4, 1e-6), device="cuda"):
    """Returns (params FP32 device tensor, losses numpy array, labels device tensor).  With
    bf16_steps > 0 every returned parameter is a BF16 value (see the module's docstring)."""
    import torch
    import paper_2302_05170_b300 as sl

    th = torch.as_tensor(np.asarray(theta, np.float32), device=device)
    yi = torch.as_tensor(np.asarray(Yi, np.float32), device=device)
    dtv = torch.as_tensor(np.asarray(dt, np.float32), device=device)
    n_rows = yi.numel()
    labels = sl.em_collocation_labels(sde, th, yi, dtv, n_paths, n_fine, m, label_seed)
    feats = torch.cat([yi[:, None], dtv[:, None], th.reshape(n_rows, -1)], 1).contiguous()
    d_in = feats.shape[1]
    P = torch.as_tensor(W.xavier_params(d_in, m, seed=init_seed), device=device)
    ws = torch.empty(sl.train_workspace_size(d_in, m, batch), dtype=torch.uint8, device=device)
    if normalize:
        f64, y64 = feats.double(), labels.double()
        fsh, ysh = f64.mean(0), y64.mean(0)
        fsc, ysc = f64.std(0), y64.std(0)
        fsc = torch.where(fsc > 0, fsc, torch.ones_like(fsc))
        ysc = torch.where(ysc > 0, ysc, torch.ones_like(ysc))
        fn = ((f64 - fsh) / fsc).float().contiguous()
        yn = ((y64 - ysh) / ysc).float().contiguous()
        losses = _adam_chunks(sl, P, d_in, m, fn, yn, n_steps, batch, lr0, lr_end, n_chunks, act, sl.PREC_FP32,
                              shuffle_seed, ws)
        P = fold_normalization(P, d_in, m, fsh, fsc, ysh, ysc)
    else:
        losses = _adam_chunks(sl, P, d_in, m, feats, labels, n_steps, batch, lr0, lr_end, n_chunks, act,
                              sl.PREC_FP32, shuffle_seed, ws)
    if bf16_steps > 0:
        losses += _adam_chunks(sl, P, d_in, m, feats, labels, bf16_steps, batch, bf16_lr[0], bf16_lr[1],
                               max(1, n_chunks // 4), act, sl.PREC_BF16, shuffle_seed + 1000, ws)
        P = P.to(torch.bfloat16).to(torch.float32)
    return P, torch.cat(losses).cpu().numpy(), labels


def train_gbm_online_network(n_rows=1 << 15, n_steps=40_000, dts=(0.125, 0.25, 0.5, 1.0), device="cuda",
                             **kw):
    """The network of the GBM online workload (d_in = 4: Y, dt, mu, sigma; m = 7), trained
    on labels for theta in [0,0.2]x[0.1,0.5], Y_i log-uniform on [0.25,4] and dt in `dts`
    (keyword arguments go to train_network)."""
    th, yi, dt = W.gbm_training_rows(n_rows, seed=2, dts=dts)
    return train_network(0, th, yi, dt, 7, n_steps=n_steps, device=device, **kw)


def train_ou_network(n_rows=1 << 14, n_steps=20_000, m=5, dts=(0.125, 0.25, 0.5, 1.0), device="cuda"):
    """The OU network of the paper's experiment (Eq. 6.5; d_in = 5: Y, dt, Ybar, sigma, lambda;
    m = 5 collocation points), trained on labels for the box of workloads.ou_training_rows."""
    th, yi, dt = W.ou_training_rows(n_rows, dts=dts)
    return train_network(1, th, yi, dt, m, n_steps=n_steps, device=device)


# --- training state on disk (weights + Adam moments + step counter) for resume -------------
STATE_VERSION = 1


def save_training_state(path, params, adam_m, adam_v, t, d_in, m, act=0):
    """Writes an .npz blob: header int64 [version, d_in, m, width, n_hidden, act, t] and the
    flat FP32 arrays params, adam_m, adam_v (layout of sl_n_params: per layer W[out][in], b)."""
    import numpy as _np

    arrs = [_np.ascontiguousarray(_np.asarray(x.detach().cpu() if hasattr(x, "detach") else x,
                                              dtype=_np.float32)) for x in (params, adam_m, adam_v)]
    n = W.n_params(d_in, m)
    if any(a.shape != (n,) for a in arrs):
        raise ValueError("state arrays must have shape (%d,)" % n)
    header = _np.array([STATE_VERSION, d_in, m, W.WIDTH, W.N_HIDDEN, act, int(t)], dtype=_np.int64)
    with open(path, "wb") as fh:
        _np.savez(fh, header=header, params=arrs[0], adam_m=arrs[1], adam_v=arrs[2])


def load_training_state(path, device=None):
    """Reads save_training_state's blob; checks the header against the arrays.  Returns a dict
    with params, adam_m, adam_v (numpy, or torch tensors on `device`), t, d_in, m, act."""
    import numpy as _np

    with _np.load(path) as z:
        header = z["header"]
        if header.shape != (7,) or int(header[0]) != STATE_VERSION:
            raise ValueError("not a training state (version %s)" % (header[:1],))
        _, d_in, m, width, n_hidden, act, t = (int(v) for v in header)
        if (width, n_hidden) != (W.WIDTH, W.N_HIDDEN):
            raise ValueError("network shape %dx%d != %dx%d" % (n_hidden, width, W.N_HIDDEN, W.WIDTH))
        n = W.n_params(d_in, m)
        out = {k: z[k].astype(_np.float32) for k in ("params", "adam_m", "adam_v")}
    for k, a in out.items():
        if a.shape != (n,):
            raise ValueError("%s has shape %s, header says (%d,)" % (k, a.shape, n))
    if device is not None:
        import torch

        out = {k: torch.as_tensor(a, device=device) for k, a in out.items()}
    out.update(t=t, d_in=d_in, m=m, act=act)
    return out
