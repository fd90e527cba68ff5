"""FP64 CPU oracle for the Seven-League scheme -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it: ``sl_oracle.c`` is written independently from the
paper's definitions (Eq. 6.2-6.6, Algorithm I) and from the published
definition of Philox4x32-10, in plain FP64 loops.

Every function is pinned by tests that do not re-use its own formulas (see the
module docstrings of ``tests/test_oracle_*.py``); none is "parity unpinned".

This module is a thin ctypes wrapper: numpy arrays in, numpy arrays out.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sl_oracle.c")
_LIB = os.path.join(_HERE, "libsl_oracle.so")

MODEL_MLP, MODEL_GBM_EXACT, MODEL_OU_EXACT = 0, 1, 2
SDE_GBM, SDE_OU, SDE_CIR = 0, 1, 2
ACT_RELU, ACT_SOFTPLUS = 0, 1
TAG_7L, TAG_EM = 0, 1
WIDTH, N_HIDDEN = 50, 4


def build(force: bool = False) -> str:
    """Compile sl_oracle.c with gcc (FP64, OpenMP) into libsl_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.POINTER(ctypes.c_int64)
_i32 = ctypes.POINTER(ctypes.c_int32)
_u32 = ctypes.POINTER(ctypes.c_uint32)
_c_int, _c_i64, _c_u32, _c_u64, _c_dbl = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                         ctypes.c_uint64, ctypes.c_double)


def _declare(L):
    L.orc_num_threads.restype = _c_int
    L.orc_philox4x32_10.argtypes = [_u32, _u32, _u32]
    L.orc_normal.argtypes = [_c_u64, _c_u32, _c_u32, _c_u32, _c_u32]
    L.orc_normal.restype = _c_dbl
    L.orc_normals.argtypes = [_c_u64, _c_u32, _c_u32, _c_u32, _c_u32, _c_int, _d]
    L.orc_gauss_hermite.argtypes = [_c_int, _d, _d]
    L.orc_gauss_hermite.restype = _c_int
    L.orc_quantile_ranks.argtypes = [_c_int, _c_i64, _i64]
    L.orc_lagrange.argtypes = [_c_int, _d, _d, _c_dbl]
    L.orc_lagrange.restype = _c_dbl
    L.orc_n_params.argtypes = [_c_int, _c_int, _c_int, _c_int]
    L.orc_n_params.restype = _c_i64
    L.orc_mlp_forward.argtypes = [_d, _c_int, _c_int, _c_int, _c_int, _c_int, _d, _c_i64, _d]
    L.orc_mse_grad.argtypes = [_d, _c_int, _c_int, _c_int, _c_int, _c_int, _d, _d, _i32, _c_i64, _d]
    L.orc_mse_grad.restype = _c_dbl
    L.orc_mlp_vjp_input.argtypes = [_d, _c_int, _c_int, _c_int, _c_int, _c_int, _d, _d, _c_i64, _d]
    L.orc_train_adam.argtypes = [_d, _d, _d, _c_i64, _c_int, _c_int, _c_int, _c_int, _c_int, _d, _d,
                                 _i32, _c_int, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _d]
    L.orc_7l_paths.argtypes = [_c_int, _d, _c_int, _c_int, _c_int, _c_int, _d, _c_int, _d, _i64,
                               _c_int, _c_dbl, _c_int, _c_int, _c_u64, _i64, _c_i64, _d, _d, _c_int]
    L.orc_7l_paths.restype = _c_int
    L.orc_7l_moments.argtypes = [_c_int, _d, _c_int, _c_int, _c_int, _c_int, _d, _c_int, _d, _i64,
                                 _c_int, _c_dbl, _c_int, _c_int, _c_u64, _d, _d, _c_int]
    L.orc_7l_moments.restype = _c_int
    L.orc_7l_payoff_grad.argtypes = [_c_int, _d, _c_int, _c_int, _c_int, _c_int, _d, _c_int, _d,
                                     _i64, _c_int, _c_dbl, _c_int, _c_int, _c_u64, _c_dbl, _i64,
                                     _c_i64, _d, _d, _d, _c_int]
    L.orc_7l_payoff_grad.restype = _c_int
    L.orc_7l_relu_margin.argtypes = [_d, _c_int, _c_int, _c_int, _d, _c_int, _d, _i64, _c_int, _c_dbl,
                                     _c_int, _c_int, _c_u64, _i64, _c_i64, _d, _c_int]
    L.orc_7l_relu_margin.restype = _c_int
    L.orc_em_terminal.argtypes = [_c_int, _d, _d, _d, _c_int, _c_int, _c_i64, _c_int, _c_u64, _d,
                                  _c_int]
    L.orc_order_statistics.argtypes = [_d, _i64, _c_int, _i64, _c_int, _d]
    L.orc_em_labels.argtypes = [_c_int, _d, _d, _d, _c_int, _c_int, _c_i64, _c_int, _c_int, _c_u64,
                                _d, _c_int]
    L.orc_em_labels.restype = _c_int
    L.orc_cdc_conditional_points.argtypes = [_c_int, _d, _d, _c_dbl, _d]
    L.orc_cdc_tables.argtypes = [_c_int, _d, _d, _c_int, _c_int, _c_int, _c_int, _d, _c_int, _d, _c_int,
                                 _c_dbl, _c_int, _c_int, _i64, _c_i64, _d, _d]
    L.orc_cdc_tables.restype = _c_int
    L.orc_cdc_paths.argtypes = [_c_int, _d, _d, _c_int, _c_int, _c_int, _c_int, _d, _c_int, _d, _i64,
                                _c_int, _c_dbl, _c_int, _c_int, _c_u64, _i64, _c_i64, _d, _d, _c_int]
    L.orc_cdc_paths.restype = _c_int
    L.orc_cdcq_G.argtypes = [_c_int, _d, _d, _c_dbl]
    L.orc_cdcq_G.restype = _c_dbl
    L.orc_cdcq_Ginv.argtypes = [_c_int, _d, _d, _c_dbl]
    L.orc_cdcq_Ginv.restype = _c_dbl
    L.orc_cdcq_F.argtypes = [_c_int, _d, _d, _c_dbl, _c_dbl]
    L.orc_cdcq_F.restype = _c_dbl
    L.orc_cdcq_tables.argtypes = [_c_int, _d, _d, _c_int, _c_int, _c_int, _c_int, _d, _c_int, _d, _c_int,
                                  _c_dbl, _c_int, _c_int, _i64, _c_i64, _d, _d]
    L.orc_cdcq_tables.restype = _c_int
    L.orc_cdcq_paths.argtypes = [_c_int, _d, _d, _c_int, _c_int, _c_int, _c_int, _d, _c_int, _d, _i64,
                                 _c_int, _c_dbl, _c_int, _c_int, _c_u64, _i64, _c_i64, _d, _d, _c_int]
    L.orc_cdcq_paths.restype = _c_int


def _p(a, ct):
    return a.ctypes.data_as(ct) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64a(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, _u32), _p(k, _u32), _p(out, _u32))
    return out


def normals(seed, tag, set_, path, first_step, n):
    out = np.zeros(n, dtype=np.float64)
    lib().orc_normals(seed, tag, set_, path, first_step, n, _p(out, _d))
    return out


def gauss_hermite(m):
    x = np.zeros(m)
    w = np.zeros(m)
    rc = lib().orc_gauss_hermite(m, _p(x, _d), _p(w, _d))
    if rc:
        raise ValueError("gauss_hermite failed for m=%d" % m)
    return x, w


def quantile_ranks(m, n):
    r = np.zeros(m, dtype=np.int64)
    lib().orc_quantile_ranks(m, n, _p(r, _i64))
    return r


def lagrange(xn, y, X):
    xn, y = _f64(xn), _f64(y)
    return float(lib().orc_lagrange(len(xn), _p(xn, _d), _p(y, _d), float(X)))


def n_params(d_in, m, width=WIDTH, n_hidden=N_HIDDEN):
    return int(lib().orc_n_params(d_in, width, n_hidden, m))


def mlp_forward(P, feats, d_in, m, act=ACT_RELU, width=WIDTH, n_hidden=N_HIDDEN):
    P, f = _f64(P), _f64(feats).reshape(-1, d_in)
    out = np.zeros((f.shape[0], m))
    lib().orc_mlp_forward(_p(P, _d), d_in, width, n_hidden, m, act, _p(f, _d), f.shape[0], _p(out, _d))
    return out


def mse_grad(P, feats, labels, d_in, m, rows=None, act=ACT_RELU, width=WIDTH, n_hidden=N_HIDDEN):
    P, f, y = _f64(P), _f64(feats).reshape(-1, d_in), _f64(labels).reshape(-1, m)
    r = None if rows is None else np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
    n = f.shape[0] if r is None else r.shape[0]
    g = np.zeros_like(P)
    loss = lib().orc_mse_grad(_p(P, _d), d_in, width, n_hidden, m, act, _p(f, _d), _p(y, _d),
                              _p(r, _i32), n, _p(g, _d))
    return float(loss), g


def mlp_vjp_input(P, feats, c, d_in, m, act=ACT_RELU, width=WIDTH, n_hidden=N_HIDDEN):
    P, f, c = _f64(P), _f64(feats).reshape(-1, d_in), _f64(c).reshape(-1, m)
    g = np.zeros_like(f)
    lib().orc_mlp_vjp_input(_p(P, _d), d_in, width, n_hidden, m, act, _p(f, _d), _p(c, _d),
                            f.shape[0], _p(g, _d))
    return g


def train_adam(P, am, av, t0, feats, labels, batch_rows, batch, d_in, m, lr=1e-3, b1=0.9,
               b2=0.999, eps=1e-8, act=ACT_RELU, width=WIDTH, n_hidden=N_HIDDEN):
    """Runs len(batch_rows)//batch Adam steps in place on copies; returns (P, am, av, losses)."""
    P, am, av = _f64(P).copy(), _f64(am).copy(), _f64(av).copy()
    f, y = _f64(feats).reshape(-1, d_in), _f64(labels).reshape(-1, m)
    br = np.ascontiguousarray(np.asarray(batch_rows, dtype=np.int32).ravel())
    nb = br.shape[0] // batch
    losses = np.zeros(nb)
    lib().orc_train_adam(_p(P, _d), _p(am, _d), _p(av, _d), t0, d_in, width, n_hidden, m, act,
                         _p(f, _d), _p(y, _d), _p(br, _i32), nb, batch, lr, b1, b2, eps,
                         _p(losses, _d))
    return P, am, av, losses


def _offsets(offsets):
    o = _i64a(offsets)
    return o, o.shape[0] - 1


def seven_league_paths(model, P, theta, Y0, offsets, T, n_steps, m, seed, idx=None, d_in=3,
                       act=ACT_RELU, grid=False, threads=0, width=WIDTH, n_hidden=N_HIDDEN):
    """Y_T (and optionally the whole grid) of selected flat paths (all if idx is None)."""
    o, n_sets = _offsets(offsets)
    th = _f64(theta).reshape(n_sets, -1)
    p = th.shape[1]
    Pp = _f64(P) if P is not None else np.zeros(1)
    y0 = _f64(Y0).reshape(n_sets)
    ix = None if idx is None else _i64a(idx)
    n = int(o[-1]) if ix is None else ix.shape[0]
    out = np.zeros(n)
    gr = np.zeros((n, n_steps + 1)) if grid else None
    rc = lib().orc_7l_paths(model, _p(Pp, _d), d_in, width, n_hidden, act, _p(th, _d), p,
                            _p(y0, _d), _p(o, _i64), n_sets, float(T), n_steps, m, seed,
                            _p(ix, _i64), n, _p(out, _d), _p(gr, _d), threads)
    if rc:
        raise ValueError("orc_7l_paths failed")
    return (out, gr) if grid else out


def seven_league_moments(model, P, theta, Y0, offsets, T, n_steps, m, seed, d_in=3,
                         act=ACT_RELU, threads=0, width=WIDTH, n_hidden=N_HIDDEN):
    o, n_sets = _offsets(offsets)
    th = _f64(theta).reshape(n_sets, -1)
    Pp = _f64(P) if P is not None else np.zeros(1)
    y0 = _f64(Y0).reshape(n_sets)
    mean, var = np.zeros(n_sets), np.zeros(n_sets)
    rc = lib().orc_7l_moments(model, _p(Pp, _d), d_in, width, n_hidden, act, _p(th, _d),
                              th.shape[1], _p(y0, _d), _p(o, _i64), n_sets, float(T), n_steps, m,
                              seed, _p(mean, _d), _p(var, _d), threads)
    if rc:
        raise ValueError("orc_7l_moments failed")
    return mean, var


def seven_league_payoff_grad(model, P, theta, Y0, offsets, T, n_steps, m, seed, K, idx=None,
                             d_in=3, act=ACT_RELU, threads=0, width=WIDTH, n_hidden=N_HIDDEN):
    """Per path: (Y_T, max(Y_T-K,0), 1{Y_T>K} dY_T/d(Y0,theta)) by forward-mode propagation."""
    o, n_sets = _offsets(offsets)
    th = _f64(theta).reshape(n_sets, -1)
    p = th.shape[1]
    Pp = _f64(P) if P is not None else np.zeros(1)
    y0 = _f64(Y0).reshape(n_sets)
    ix = None if idx is None else _i64a(idx)
    n = int(o[-1]) if ix is None else ix.shape[0]
    yt, val, gr = np.zeros(n), np.zeros(n), np.zeros((n, 1 + p))
    rc = lib().orc_7l_payoff_grad(model, _p(Pp, _d), d_in, width, n_hidden, act, _p(th, _d), p,
                                  _p(y0, _d), _p(o, _i64), n_sets, float(T), n_steps, m, seed,
                                  float(K), _p(ix, _i64), n, _p(yt, _d), _p(val, _d), _p(gr, _d),
                                  threads)
    if rc:
        raise ValueError("orc_7l_payoff_grad failed")
    return yt, val, gr


def seven_league_relu_margin(P, theta, Y0, offsets, T, n_steps, m, seed, idx=None, d_in=3, threads=0,
                             width=WIDTH, n_hidden=N_HIDDEN):
    """Per selected path: min |hidden pre-activation| over the network evaluations
    along the path (the distance of its ReLU pattern from a switch)."""
    o, n_sets = _offsets(offsets)
    th = _f64(theta).reshape(n_sets, -1)
    y0 = _f64(Y0).reshape(n_sets)
    ix = None if idx is None else _i64a(idx)
    n = int(o[-1]) if ix is None else ix.shape[0]
    out = np.zeros(n)
    rc = lib().orc_7l_relu_margin(_p(_f64(P), _d), d_in, width, n_hidden, _p(th, _d), th.shape[1],
                                  _p(y0, _d), _p(o, _i64), n_sets, float(T), n_steps, m, seed,
                                  _p(ix, _i64), n, _p(out, _d), threads)
    if rc:
        raise ValueError("orc_7l_relu_margin failed")
    return out


def em_terminal(sde, theta, Yi, dt, n_paths, n_fine, seed, row0=0, n_rows=None, threads=0):
    th = _f64(theta)
    yi, dtv = _f64(Yi).ravel(), _f64(dt).ravel()
    n_rows = yi.shape[0] - row0 if n_rows is None else n_rows
    out = np.zeros((n_rows, n_paths))
    lib().orc_em_terminal(sde, _p(th, _d), _p(yi, _d), _p(dtv, _d), row0, n_rows, n_paths, n_fine,
                          seed, _p(out, _d), threads)
    return out


def order_statistics(values, seg_off, ranks):
    v, o, r = _f64(values), _i64a(seg_off), _i64a(ranks)
    out = np.zeros((o.shape[0] - 1, r.shape[0]))
    lib().orc_order_statistics(_p(v, _d), _p(o, _i64), o.shape[0] - 1, _p(r, _i64), r.shape[0],
                               _p(out, _d))
    return out


def em_labels(sde, theta, Yi, dt, n_paths, n_fine, m, seed, row0=0, n_rows=None, threads=0):
    th = _f64(theta)
    yi, dtv = _f64(Yi).ravel(), _f64(dt).ravel()
    n_rows = yi.shape[0] - row0 if n_rows is None else n_rows
    out = np.zeros((n_rows, m))
    rc = lib().orc_em_labels(sde, _p(th, _d), _p(yi, _d), _p(dtv, _d), row0, n_rows, n_paths,
                             n_fine, m, seed, _p(out, _d), threads)
    if rc:
        raise ValueError("orc_em_labels failed")
    return out


# --- the 7L-CDC variant (global interpolation in Y through marginal collocation points) ----
def cdc_conditional_points(z, C, Y):
    """yhat_j = sum_k C[k, j] L_k(Y), L_k the Lagrange basis through the nodes z (row 0
    when all nodes coincide)."""
    zz = _f64(z)
    m = zz.shape[0]
    CC = _f64(C).reshape(m, m)
    out = np.zeros(m)
    lib().orc_cdc_conditional_points(m, _p(zz, _d), _p(CC, _d), float(Y), _p(out, _d))
    return out


def cdc_tables(model, P, theta, Y0, T, n_steps, m, Pm=None, d_in=3, act=ACT_RELU, width=WIDTH,
               n_hidden=N_HIDDEN, sets=None):
    """Marginal nodes z [n, n_steps, m] and conditional points at them C [n, n_steps, m (node k),
    m (point j)] for the sets `sets` (row r = set sets[r]; None: every set, n = n_sets)."""
    y0 = _f64(Y0).reshape(-1)
    n_sets = y0.shape[0]
    th = _f64(theta).reshape(n_sets, -1)
    Pp = _f64(P) if P is not None else np.zeros(1)
    Pmp = _f64(Pm) if Pm is not None else None
    sel = None if sets is None else _i64a(sets)
    n = n_sets if sel is None else sel.shape[0]
    z = np.zeros((n, n_steps, m))
    C = np.zeros((n, n_steps, m, m))
    rc = lib().orc_cdc_tables(model, _p(Pp, _d), _p(Pmp, _d), d_in, width, n_hidden, act, _p(th, _d),
                              th.shape[1], _p(y0, _d), n_sets, float(T), n_steps, m, _p(sel, _i64),
                              0 if sel is None else n, _p(z, _d), _p(C, _d))
    if rc:
        raise ValueError("orc_cdc_tables failed")
    return z, C


def cdc_paths(model, P, theta, Y0, offsets, T, n_steps, m, seed, Pm=None, idx=None, d_in=3,
              act=ACT_RELU, grid=False, threads=0, width=WIDTH, n_hidden=N_HIDDEN):
    """Y_T (and optionally the grid) of selected flat paths of the 7L-CDC chain."""
    o, n_sets = _offsets(offsets)
    th = _f64(theta).reshape(n_sets, -1)
    Pp = _f64(P) if P is not None else np.zeros(1)
    Pmp = _f64(Pm) if Pm is not None else None
    y0 = _f64(Y0).reshape(n_sets)
    ix = None if idx is None else _i64a(idx)
    n = int(o[-1]) if ix is None else ix.shape[0]
    out = np.zeros(n)
    gr = np.zeros((n, n_steps + 1)) if grid else None
    rc = lib().orc_cdc_paths(model, _p(Pp, _d), _p(Pmp, _d), d_in, width, n_hidden, act, _p(th, _d),
                             th.shape[1], _p(y0, _d), _p(o, _i64), n_sets, float(T), n_steps, m, seed,
                             _p(ix, _i64), n, _p(out, _d), _p(gr, _d), threads)
    if rc:
        raise ValueError("orc_cdc_paths failed")
    return (out, gr) if grid else out


# --- the 7L-CDC variant in the marginal's quantile coordinate -------------------------------
def _gh_nodes(m):
    xn, wn = np.zeros(64), np.zeros(64)
    lib().orc_gauss_hermite(m, _p(xn, _d), _p(wn, _d))
    return xn[:m].copy()


def cdcq_G(z, xi):
    """G(xi) through (x_k, z_k) at the Gauss-Hermite points, continued linearly."""
    zz = _f64(z)
    m = zz.shape[0]
    xn = _gh_nodes(m)
    return lib().orc_cdcq_G(m, _p(xn, _d), _p(zz, _d), float(xi))


def cdcq_Ginv(z, y):
    zz = _f64(z)
    m = zz.shape[0]
    xn = _gh_nodes(m)
    return lib().orc_cdcq_Ginv(m, _p(xn, _d), _p(zz, _d), float(y))


def cdcq_F(eta, xi, X):
    """sum_k sum_j eta[k, j] L_k(xi) L_j(X) at the Gauss-Hermite points."""
    e = _f64(eta)
    m = e.shape[0]
    xn = _gh_nodes(m)
    return lib().orc_cdcq_F(m, _p(xn, _d), _p(e, _d), float(xi), float(X))


def cdcq_tables(model, P, theta, Y0, T, n_steps, m, Pm=None, d_in=3, act=ACT_RELU, width=WIDTH,
                n_hidden=N_HIDDEN, sets=None):
    """Nodes of t_{i+1} zn [n, n_steps, m] and eta [n, n_steps, m (node k), m (point j)]."""
    y0 = _f64(Y0).reshape(-1)
    n_sets = y0.shape[0]
    th = _f64(theta).reshape(n_sets, -1)
    Pp = _f64(P) if P is not None else np.zeros(1)
    Pmp = _f64(Pm) if Pm is not None else None
    sel = None if sets is None else _i64a(sets)
    n = n_sets if sel is None else sel.shape[0]
    zn = np.zeros((n, n_steps, m))
    eta = np.zeros((n, n_steps, m, m))
    rc = lib().orc_cdcq_tables(model, _p(Pp, _d), _p(Pmp, _d), d_in, width, n_hidden, act, _p(th, _d),
                               th.shape[1], _p(y0, _d), n_sets, float(T), n_steps, m, _p(sel, _i64),
                               0 if sel is None else n, _p(zn, _d), _p(eta, _d))
    if rc:
        raise ValueError("orc_cdcq_tables failed")
    return zn, eta


def cdcq_paths(model, P, theta, Y0, offsets, T, n_steps, m, seed, Pm=None, idx=None, d_in=3,
               act=ACT_RELU, grid=False, threads=0, width=WIDTH, n_hidden=N_HIDDEN):
    """Y_T (and optionally the grid) of selected flat paths of the quantile-coordinate chain."""
    o, n_sets = _offsets(offsets)
    th = _f64(theta).reshape(n_sets, -1)
    Pp = _f64(P) if P is not None else np.zeros(1)
    Pmp = _f64(Pm) if Pm is not None else None
    y0 = _f64(Y0).reshape(n_sets)
    ix = None if idx is None else _i64a(idx)
    n = int(o[-1]) if ix is None else ix.shape[0]
    out = np.zeros(n)
    gr = np.zeros((n, n_steps + 1)) if grid else None
    rc = lib().orc_cdcq_paths(model, _p(Pp, _d), _p(Pmp, _d), d_in, width, n_hidden, act, _p(th, _d),
                              th.shape[1], _p(y0, _d), _p(o, _i64), n_sets, float(T), n_steps, m, seed,
                              _p(ix, _i64), n, _p(out, _d), _p(gr, _d), threads)
    if rc:
        raise ValueError("orc_cdcq_paths failed")
    return (out, gr) if grid else out
