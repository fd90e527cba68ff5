"""Seeded synthetic inputs for the Seven-League hot path.

This module holds NONE of the method's arithmetic: it only draws the inputs a
user would supply -- network parameters (Glorot/Xavier-uniform, the
initialisation named in the paper's experiments section), parameter sets
theta, start values, per-set path counts, training rows and minibatch orders.
The normal draws X of the method itself are NOT made here; both the CUDA
library and the oracle derive them from the counter-based Philox4x32-10
stream keyed by the call's seed.

Every generator takes an explicit seed and uses numpy's PCG64, so the test
suite, the benchmark and a user can reproduce the same inputs.

Workloads (the shapes used by tests and the benchmark):
  * GBM_SMALL   -- GBM mu=0.1, sigma=0.3, Y0=1, T=1, 2 coarse steps, m=5,
                   MLP 3->50x4->5 ReLU, Xavier seed 0, 10^4 paths, seed 1.
  * GBM_ONLINE  -- 16 theta=(mu, sigma) ~ U([0,0.2]x[0.1,0.5]), Y0=1, T=2,
                   16 coarse steps, m=7, MLP 4->50x4->7, 10^6 paths per theta.
  * CIR_LABELS  -- 1024 rows (kappa, ybar, gamma, Y_i, dt) uniform in
                   [0.5,2]x[0.05,0.3]x[0.1,0.5]x[0.01,0.5]x[0.1,1],
                   10^5 EM paths each, 100 fine steps, 7 quantiles.
  * CIR_BATCHED -- 4096 CIR theta sets from the same box, per-set path
                   counts round(10^(3+2u)), Y0=0.1, dt=0.25, 32 steps, m=7.
  * ADJOINT     -- GBM (mu=0.1, sigma=0.3, Y0=1, T=1) and CIR (kappa=1,
                   ybar=0.1, gamma=0.3, Y0=0.1), 10^6 paths, 64 steps, m=7.
"""
from __future__ import annotations

import numpy as np

WIDTH = 50
N_HIDDEN = 4


def n_params(d_in: int, m: int, width: int = WIDTH, n_hidden: int = N_HIDDEN) -> int:
    return width * d_in + width + (n_hidden - 1) * (width * width + width) + m * width + m


def layer_shapes(d_in: int, m: int, width: int = WIDTH, n_hidden: int = N_HIDDEN):
    """(out, in) of every layer, input layer first."""
    shapes = [(width, d_in)] + [(width, width)] * (n_hidden - 1) + [(m, width)]
    return shapes


def xavier_params(d_in: int, m: int, seed: int = 0, width: int = WIDTH,
                  n_hidden: int = N_HIDDEN) -> np.ndarray:
    """Flat FP32 parameters: per layer W (row-major [out][in]) then b.

    W ~ U(-a, a), a = sqrt(6 / (fan_in + fan_out)) (Glorot & Bengio 2010);
    biases are zero.
    """
    rng = np.random.default_rng(seed)
    parts = []
    for (fo, fi) in layer_shapes(d_in, m, width, n_hidden):
        a = np.sqrt(6.0 / (fi + fo))
        parts.append(rng.uniform(-a, a, size=fo * fi))
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def near_affine_params(d_in: int, m: int, a: float = 0.2, b: float = 0.3, eps: float = 0.02,
                       seed: int = 0, shift: float = 1.5) -> np.ndarray:
    """A network whose outputs look like collocation points, for the 7L-CDC variant (whose
    marginal points an untrained network leaves unordered or nearly coincident).

    Before the perturbation it computes y_j = Y + x_j (a + b dt) exactly (x_j the ascending
    Gauss-Hermite points of N(0,1), from numpy) while every feature exceeds -shift: hidden
    units u < d_in carry feature u + shift through every layer (on the linear side of the
    ReLU), the other units are zero, and the output layer undoes the shift.  A small shift
    keeps the output from being a difference of large terms (FP32 evaluations stay accurate).  Then eps times Xavier-uniform
    weights (seed) are added to every weight, so some units switch and the map is no
    longer affine.
    """
    from numpy.polynomial import hermite_e

    x = hermite_e.hermegauss(m)[0]
    parts = []
    for li, (fo, fi) in enumerate(layer_shapes(d_in, m)):
        Wl = np.zeros((fo, fi))
        bl = np.zeros(fo)
        if li < N_HIDDEN:
            for u in range(d_in):
                Wl[u, u] = 1.0
            if li == 0:
                bl[:d_in] = shift
        else:
            Wl[:, 0] = 1.0
            Wl[:, 1] = b * x
            bl[:] = a * x - shift * (1.0 + b * x)
        parts += [Wl.ravel(), bl]
    P = np.concatenate(parts)
    return (P + eps * xavier_params(d_in, m, seed=seed).astype(np.float64)).astype(np.float32)


def split_params(P: np.ndarray, d_in: int, m: int, width: int = WIDTH, n_hidden: int = N_HIDDEN):
    """Views [(W, b), ...] of a flat parameter array."""
    out, o = [], 0
    for (fo, fi) in layer_shapes(d_in, m, width, n_hidden):
        W = P[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = P[o:o + fo]
        o += fo
        out.append((W, b))
    return out


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 value (ties to even), returned as FP32."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def offsets_from_counts(counts) -> np.ndarray:
    c = np.asarray(counts, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(c)]).astype(np.int64)


# --------------------------------------------------------------------------
# GBM_SMALL: one theta set.  The network of this workload has d_in = 3, so it
# sees theta = (sigma) besides (Y_i, dt); mu = 0.1 is a constant of the model.
# --------------------------------------------------------------------------
def gbm_small(n_paths: int = 10_000):
    return dict(model="mlp", d_in=3, m=5, theta=np.array([[0.3]], dtype=np.float32),
                Y0=np.array([1.0], dtype=np.float32), offsets=offsets_from_counts([n_paths]),
                T=1.0, n_steps=2, seed=1, params=xavier_params(3, 5, seed=0))


def gbm_online_thetas(n_sets: int = 16, seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.0, 0.2, n_sets)
    sg = rng.uniform(0.1, 0.5, n_sets)
    return np.stack([mu, sg], axis=1).astype(np.float32)


def gbm_online(n_paths_per_set: int = 1_000_000, n_sets: int = 16, params=None):
    th = gbm_online_thetas(n_sets)
    return dict(model="mlp", d_in=4, m=7, theta=th, Y0=np.ones(n_sets, dtype=np.float32),
                offsets=offsets_from_counts([n_paths_per_set] * n_sets), T=2.0, n_steps=16,
                seed=1, params=params if params is not None else xavier_params(4, 7, seed=0))


def gbm_training_rows(n_rows: int, seed: int = 2, dt: float = 0.125, dts=None):
    """Training rows (theta=(mu,sigma), Y_i, dt) for the GBM network of GBM_ONLINE:
    mu ~ U[0,0.2], sigma ~ U[0.1,0.5], Y_i log-uniform on [0.25, 4]; dt fixed, or
    drawn uniformly from the values `dts`."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.0, 0.2, n_rows)
    sg = rng.uniform(0.1, 0.5, n_rows)
    yi = np.exp(rng.uniform(np.log(0.25), np.log(4.0), n_rows))
    dtv = np.full(n_rows, dt) if dts is None else rng.choice(np.asarray(dts, np.float64), n_rows)
    return (np.stack([mu, sg], 1).astype(np.float32), yi.astype(np.float32), dtv.astype(np.float32))


def ou_training_rows(n_rows: int, seed: int = 12, dts=(0.125, 0.25, 0.5, 1.0)):
    """Training rows (theta=(Ybar, sigma, lambda), Y_i, dt) for the OU network of the
    paper's experiment (Eq. 6.5): Ybar ~ U[0,1], sigma ~ U[0.1,0.5], lambda ~ U[0.5,2],
    Y_i ~ U[-1,2], dt drawn uniformly from `dts`."""
    rng = np.random.default_rng(seed)
    yb = rng.uniform(0.0, 1.0, n_rows)
    sg = rng.uniform(0.1, 0.5, n_rows)
    lam = rng.uniform(0.5, 2.0, n_rows)
    yi = rng.uniform(-1.0, 2.0, n_rows)
    dtv = rng.choice(np.asarray(dts, np.float64), n_rows)
    return (np.stack([yb, sg, lam], 1).astype(np.float32), yi.astype(np.float32), dtv.astype(np.float32))


def cir_label_rows(n_rows: int = 1024, seed: int = 3):
    """CIR_LABELS rows: theta=(kappa, ybar, gamma), Y_i, dt uniform in their boxes."""
    rng = np.random.default_rng(seed)
    kappa = rng.uniform(0.5, 2.0, n_rows)
    ybar = rng.uniform(0.05, 0.3, n_rows)
    gamma = rng.uniform(0.1, 0.5, n_rows)
    yi = rng.uniform(0.01, 0.5, n_rows)
    dt = rng.uniform(0.1, 1.0, n_rows)
    return (np.stack([kappa, ybar, gamma], 1).astype(np.float32), yi.astype(np.float32),
            dt.astype(np.float32))


def cir_batched(n_sets: int = 4096, seed: int = 4, lo_exp: float = 3.0, hi_exp: float = 5.0):
    """CIR_BATCHED: theta sets from the CIR box and log-uniform path counts."""
    rng = np.random.default_rng(seed)
    kappa = rng.uniform(0.5, 2.0, n_sets)
    ybar = rng.uniform(0.05, 0.3, n_sets)
    gamma = rng.uniform(0.1, 0.5, n_sets)
    counts = np.rint(10.0 ** rng.uniform(lo_exp, hi_exp, n_sets)).astype(np.int64)
    return dict(theta=np.stack([kappa, ybar, gamma], 1).astype(np.float32),
                Y0=np.full(n_sets, 0.1, dtype=np.float32), offsets=offsets_from_counts(counts),
                T=8.0, n_steps=32, seed=1, m=7, d_in=5)


def minibatch_rows(n_rows: int, batch: int, n_batches: int, seed: int = 5) -> np.ndarray:
    """Row indices of n_batches minibatches: consecutive epochs of random permutations."""
    rng = np.random.default_rng(seed)
    need = batch * n_batches
    out = []
    while sum(len(o) for o in out) < need:
        out.append(rng.permutation(n_rows))
    return np.concatenate(out)[:need].astype(np.int32).reshape(n_batches, batch)


def random_segments(n_seg: int, max_len: int, seed: int = 6, ties: bool = False):
    """Float segments of ragged lengths (0..max_len) for order-statistic tests."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len + 1, n_seg)
    if n_seg > 2:
        lens[0], lens[1] = 0, 1
    off = offsets_from_counts(lens)
    n = int(off[-1])
    if ties:
        v = rng.integers(-20, 20, n).astype(np.float32) * 0.25
    else:
        v = (rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))).astype(np.float32)
    return v, off
