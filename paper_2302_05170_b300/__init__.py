"""B300-native Seven-League (7L) library: Python binding of libsevenleague.so.

The functions below have the names of the C ABI entry points in
``include/sevenleague.h`` and only marshal arguments: torch CUDA tensors are
passed as device pointers together with the current CUDA stream, and scratch
buffers are allocated with torch (PyTorch is used for device memory and
streams only).  Every step of the computation runs in the library's kernels;
there is no CPU fallback -- if the shared library is missing or no GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads  # noqa: F401  (seeded synthetic inputs)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsevenleague.so")
# the same library built with -DSL_CHECKED: kernels verify device-derived indices (a path's
# set against path_offsets, listed paths against the path count) and report SL_DEV_OFFSETS /
# SL_DEV_INDEX instead of trusting them; load(LIB_CHECKED_PATH) in a process of its own
LIB_CHECKED_PATH = os.path.join(_HERE, "libsevenleague_checked.so")

# Codes of include/sevenleague.h
SL_OK, SL_ERR_ARG, SL_ERR_UNSUPPORTED, SL_ERR_WORKSPACE, SL_ERR_CUDA, SL_ERR_DEVICE, SL_ERR_TIMEOUT = range(7)
MODEL_MLP, MODEL_GBM_EXACT, MODEL_OU_EXACT = 0, 1, 2
SDE_GBM, SDE_OU, SDE_CIR = 0, 1, 2
ACT_RELU, ACT_SOFTPLUS = 0, 1
PREC_FP32, PREC_BF16 = 0, 1
PAYOFF_CALL = 0
CDC_Y, CDC_QUANTILE = 0, 1          # 7L-CDC interpolation space (SL_CDC_SPACE_*)
WIDTH, N_HIDDEN, MIN_M, MAX_M = 50, 4, 2, 8
SL_DEV_NONFINITE, SL_DEV_OFFSETS, SL_DEV_TIMEOUT, SL_DEV_INDEX = 0x1, 0x2, 0x4, 0x8   # device status bits
_STATUS_NAMES = {1: "SL_ERR_ARG", 2: "SL_ERR_UNSUPPORTED", 3: "SL_ERR_WORKSPACE",
                 4: "SL_ERR_CUDA", 5: "SL_ERR_DEVICE", 6: "SL_ERR_TIMEOUT"}

# Every symbol the header declares (checked by the test suite without a GPU).
EXPORTED = [
    "sl_version", "sl_last_error_string", "sl_n_params", "sl_gauss_hermite",
    "sl_quantile_ranks", "sl_workspace_status", "sl_simulate_workspace_size",
    "seven_league_simulate_batched", "seven_league_simulate", "sl_em_terminal",
    "sl_select_workspace_size", "sl_segmented_select", "sl_em_labels_workspace_size",
    "em_collocation_labels", "sl_tc_set_slots", "sl_tc_get_slots", "sl_tc_set_pipeline",
    "sl_tc_get_pipeline", "sl_train_workspace_size",
    "sl_mlp_forward", "sl_mse_grad", "sl_adam_step", "sl_train", "sl_adjoint_workspace_size",
    "seven_league_adjoint", "em_collocation_labels_noalloc", "sl_em_labels_noalloc_max_samples",
    "sl_selftest_wait_timeout", "sl_cdc_workspace_size", "seven_league_cdc_simulate_batched",
    "sl_cdcq_inverse", "sl_simulate_range_workspace_size", "seven_league_simulate_range",
]


class SLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, status), msg))
        self.status = status


class sl_net(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("d_in", ctypes.c_int), ("m", ctypes.c_int),
                ("act", ctypes.c_int), ("prec", ctypes.c_int)]


_lib = None
_vp, _i, _i64, _u64, _f, _sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                 ctypes.c_float, ctypes.c_size_t)


from . import build as _build_module   # noqa: E402  (the submodule; `build` below is the function)


def build(verbose: bool = False, checked: bool = False) -> str:
    """Compile the CUDA sources for sm_103a (nvcc) into the in-tree library (checked=True:
    the checked build, libsevenleague_checked.so)."""
    return _build_module.build(verbose=verbose, checked=checked)


def load(path: str = LIB_PATH):
    """Load libsevenleague.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsevenleague.so not built (%s); run paper_2302_05170_b300.build()" % path)
    L = ctypes.CDLL(path)
    L.sl_version.restype = _i
    L.sl_last_error_string.restype = ctypes.c_char_p
    L.sl_n_params.argtypes = [_i, _i]
    L.sl_n_params.restype = _i64
    L.sl_gauss_hermite.argtypes = [_i, _vp, _vp, _vp]
    L.sl_quantile_ranks.argtypes = [_i, _i64, _vp]
    L.sl_workspace_status.argtypes = [_vp, _vp, _vp]
    L.sl_simulate_workspace_size.argtypes = [_i64, _i]
    L.sl_simulate_workspace_size.restype = _sz
    L.seven_league_simulate_batched.argtypes = [
        _i, ctypes.POINTER(sl_net), _vp, _i, _vp, _vp, _i, _i64, _f, _i, _i, _u64,
        _vp, _vp, _vp, _vp, _vp, _sz, _vp]
    L.seven_league_simulate.argtypes = [_i, _vp, _i, _f, _f, _i, _i, ctypes.POINTER(sl_net), _i64,
                                        _u64, _vp, _vp]
    L.sl_simulate_range_workspace_size.argtypes = [_i64, _i]
    L.sl_simulate_range_workspace_size.restype = _sz
    L.seven_league_simulate_range.argtypes = [
        _i, ctypes.POINTER(sl_net), _vp, _i, _vp, _vp, _i, _i64, _i64, _f, _i, _i, _u64,
        _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
    L.sl_em_terminal.argtypes = [_i, _vp, _vp, _vp, _i, _i64, _i, _u64, _vp, _vp]
    L.sl_select_workspace_size.argtypes = [_i, _i]
    L.sl_select_workspace_size.restype = _sz
    L.sl_segmented_select.argtypes = [_vp, _vp, _i, _vp, _i, _vp, _vp, _sz, _vp]
    L.sl_em_labels_workspace_size.argtypes = [_i, _i64, _i]
    L.sl_em_labels_workspace_size.restype = _sz
    L.em_collocation_labels.argtypes = [_i, _vp, _vp, _vp, _i, _i64, _i, _i, _u64, _vp, _vp, _sz, _vp]
    L.sl_train_workspace_size.argtypes = [_i, _i, _i]
    L.sl_train_workspace_size.restype = _sz
    L.sl_mlp_forward.argtypes = [ctypes.POINTER(sl_net), _vp, _i64, _vp, _vp]
    L.sl_mse_grad.argtypes = [ctypes.POINTER(sl_net), _vp, _vp, _vp, _i, _vp, _vp, _vp, _sz, _vp]
    L.sl_adam_step.argtypes = [_vp, _vp, _vp, _vp, _i64, _i64, _f, _f, _f, _f, _vp]
    L.sl_train.argtypes = [_vp, _i, _i, _i, _i, _vp, _vp, _i64, _vp, _vp, _vp, _i, _i, _f, _f, _f, _f,
                           _vp, _vp, _sz, _vp]
    L.sl_adjoint_workspace_size.argtypes = [_i64, _i, _i, _i, _i]
    L.sl_adjoint_workspace_size.restype = _sz
    L.seven_league_adjoint.argtypes = [_i, ctypes.POINTER(sl_net), _vp, _i, _vp, _vp, _i, _i64, _f, _i, _i,
                                       _u64, _i, _f, _i, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
    L.sl_selftest_wait_timeout.argtypes = [_vp, _sz, _vp]
    L.sl_cdc_workspace_size.argtypes = [_i64, _i, _i]
    L.sl_cdc_workspace_size.restype = _sz
    L.seven_league_cdc_simulate_batched.argtypes = [
        _i, ctypes.POINTER(sl_net), ctypes.POINTER(sl_net), _i, _vp, _i, _vp, _vp, _i, _i64, _f, _i, _i, _u64,
        _vp, _vp, _vp, _vp, _vp, _sz, _vp]
    L.em_collocation_labels_noalloc.argtypes = [_i, _vp, _vp, _vp, _i, _i64, _i, _i, _u64, _vp, _vp]
    L.sl_cdcq_inverse.argtypes = [_i, _vp, _i, _vp, _i, _vp, _vp]
    L.sl_em_labels_noalloc_max_samples.restype = _sz
    L.sl_tc_set_pipeline.argtypes = [_i]
    L.sl_tc_get_pipeline.restype = _i
    L.sl_tc_set_slots.argtypes = [_i]
    L.sl_tc_get_slots.restype = _i
    _lib = L
    return L


def _check(rc):
    if rc != SL_OK:
        raise SLError(rc, _lib.sl_last_error_string().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (no CPU fallback)")
    return torch


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def make_net(params, d_in, m, act=ACT_RELU, prec=PREC_FP32):
    """sl_net descriptor for a device FP32 parameter tensor.  The descriptor keeps
    a reference to the tensor, so its memory stays valid while the descriptor lives."""
    torch = _torch()
    _ptr(params, torch.float32, "params")
    if params.numel() != n_params(d_in, m):
        raise ValueError("params has %d values, the network needs %d" % (params.numel(), n_params(d_in, m)))
    net = sl_net(params.data_ptr(), d_in, m, act, prec)
    net._params = params
    return net


# ---------------------------------------------------------------------------
# Host helpers
# ---------------------------------------------------------------------------
def version():
    return load().sl_version()


def n_params(d_in, m):
    return int(load().sl_n_params(d_in, m))


def gauss_hermite(m):
    L = load()
    x, w, b = np.zeros(m), np.zeros(m), np.zeros(m)
    _check(L.sl_gauss_hermite(m, x.ctypes.data, w.ctypes.data, b.ctypes.data))
    return x, w, b


def quantile_ranks(m, n):
    L = load()
    r = np.zeros(m, dtype=np.int64)
    _check(L.sl_quantile_ranks(m, n, r.ctypes.data))
    return r


def workspace_status(ws, stream=None):
    """Synchronises and returns the device status bits of a workspace."""
    L = load()
    bits = ctypes.c_uint32(0)
    rc = L.sl_workspace_status(_ptr(ws), _stream(stream), ctypes.byref(bits))
    if rc not in (SL_OK, SL_ERR_DEVICE, SL_ERR_TIMEOUT):
        _check(rc)
    return int(bits.value)


def selftest_wait_timeout(ws=None, stream=None):
    """Runs the bounded-wait self-test on the status word of `ws` (allocated if None) and
    returns the workspace (read it with workspace_status)."""
    torch = _torch()
    L = load()
    if ws is None:
        ws = _workspace(256, torch.device("cuda"))
    _check(L.sl_selftest_wait_timeout(_ptr(ws), ws.numel(), _stream(stream)))
    return ws


def tc_set_slots(slots):
    """Path tiles in flight per CTA of the BF16 tensor-core form (2..4)."""
    _check(load().sl_tc_set_slots(int(slots)))


def tc_get_slots():
    return int(load().sl_tc_get_slots())


def tc_set_pipeline(tiles_per_warpgroup):
    """Tiles per warpgroup of the BF16 form: 1 (default) or 2 (ping-pong)."""
    _check(load().sl_tc_set_pipeline(int(tiles_per_warpgroup)))


def tc_get_pipeline():
    return int(load().sl_tc_get_pipeline())


# ---------------------------------------------------------------------------
# Online stage
# ---------------------------------------------------------------------------
def simulate_workspace_size(total_paths, n_sets):
    return int(load().sl_simulate_workspace_size(total_paths, n_sets))


def seven_league_simulate_batched(model, net, theta, Y0, path_offsets, T, n_steps, m, seed,
                                  out_YT=None, out_grid=None, out_mean=None, out_var=None,
                                  ws=None, total_paths=None, stream=None):
    """Batched 7L sampler (see include/sevenleague.h).  Tensors on the GPU.
    Returns the workspace used (its first word is the device status)."""
    torch = _torch()
    L = load()
    n_sets = path_offsets.numel() - 1
    p = theta.shape[1] if theta.dim() == 2 else theta.numel() // max(n_sets, 1)
    if total_paths is None:
        total_paths = int(path_offsets[-1].item())
    if ws is None:
        ws = _workspace(L.sl_simulate_workspace_size(total_paths, n_sets), theta.device)
    netp = ctypes.byref(net) if net is not None else None
    _check(L.seven_league_simulate_batched(
        model, netp, _ptr(theta, torch.float32, "theta"), p, _ptr(Y0, torch.float32, "Y0"),
        _ptr(path_offsets, torch.int64, "path_offsets"), n_sets, int(total_paths), float(T),
        n_steps, m, seed, _ptr(out_YT, torch.float32, "out_YT"),
        _ptr(out_grid, torch.float32, "out_grid"), _ptr(out_mean, torch.float64, "out_mean"),
        _ptr(out_var, torch.float64, "out_var"), _ptr(ws), ws.numel(), _stream(stream)))
    return ws


def simulate_range_workspace_size(n_paths, n_sets):
    return int(load().sl_simulate_range_workspace_size(int(n_paths), n_sets))


def seven_league_simulate_range(model, net, theta, Y0, path_offsets, T, n_steps, m, seed, first_path, n_paths,
                                out_YT=None, out_grid=None, out_mean=None, out_var=None, out_count=None,
                                ws=None, stream=None):
    """Flat paths first_path .. first_path + n_paths - 1 of the batch that theta, Y0 and
    path_offsets describe (see include/sevenleague.h): the same per-path values as the whole
    batched call, plus per-set count / mean / variance over the range.  Returns the workspace."""
    torch = _torch()
    L = load()
    n_sets = path_offsets.numel() - 1
    p = theta.shape[1] if theta.dim() == 2 else theta.numel() // max(n_sets, 1)
    if ws is None:
        ws = _workspace(L.sl_simulate_range_workspace_size(int(n_paths), n_sets), theta.device)
    netp = ctypes.byref(net) if net is not None else None
    _check(L.seven_league_simulate_range(
        model, netp, _ptr(theta, torch.float32, "theta"), p, _ptr(Y0, torch.float32, "Y0"),
        _ptr(path_offsets, torch.int64, "path_offsets"), n_sets, int(first_path), int(n_paths), float(T),
        n_steps, m, seed, _ptr(out_YT, torch.float32, "out_YT"), _ptr(out_grid, torch.float32, "out_grid"),
        _ptr(out_mean, torch.float64, "out_mean"), _ptr(out_var, torch.float64, "out_var"),
        _ptr(out_count, torch.int64, "out_count"), _ptr(ws), ws.numel(), _stream(stream)))
    return ws


def seven_league_simulate(model, theta, Y0, T, n_steps, m, weights, n_paths, seed, out,
                          stream=None):
    """Single parameter set: theta device FP32 [p], Y0 a Python float, out [n_paths]."""
    torch = _torch()
    L = load()
    netp = ctypes.byref(weights) if weights is not None else None
    _check(L.seven_league_simulate(model, _ptr(theta, torch.float32, "theta"), theta.numel(),
                                   float(Y0), float(T), n_steps, m, netp, int(n_paths), seed,
                                   _ptr(out, torch.float32, "out"), _stream(stream)))
    return out


CDC_TABLE_FLOATS = 224  # per (set, step): z | w | C | S_lo | S_hi | C_lo | C_hi | z_lo, z_hi | D | A | B_lo | Sm_lo | B_hi | Sm_hi


def cdc_workspace_size(total_paths, n_sets, n_steps):
    return int(load().sl_cdc_workspace_size(total_paths, n_sets, n_steps))


def seven_league_cdc_simulate_batched(model, net, theta, Y0, path_offsets, T, n_steps, m, seed,
                                      marg_net=None, space=CDC_QUANTILE, out_YT=None, out_grid=None,
                                      out_mean=None, out_var=None, ws=None, total_paths=None, stream=None):
    """Batched 7L-CDC sampler (see include/sevenleague.h); marg_net None = net; space CDC_QUANTILE
    (the marginal's quantile coordinate) or CDC_Y (interpolation in Y).
    Returns the workspace used (status word first, then the tables)."""
    torch = _torch()
    L = load()
    n_sets = path_offsets.numel() - 1
    p = theta.shape[1] if theta.dim() == 2 else theta.numel() // max(n_sets, 1)
    if total_paths is None:
        total_paths = int(path_offsets[-1].item())
    if ws is None:
        ws = _workspace(L.sl_cdc_workspace_size(total_paths, n_sets, n_steps), theta.device)
    netp = ctypes.byref(net) if net is not None else None
    mnetp = ctypes.byref(marg_net) if marg_net is not None else None
    _check(L.seven_league_cdc_simulate_batched(
        model, netp, mnetp, int(space), _ptr(theta, torch.float32, "theta"), p, _ptr(Y0, torch.float32, "Y0"),
        _ptr(path_offsets, torch.int64, "path_offsets"), n_sets, int(total_paths), float(T),
        n_steps, m, seed, _ptr(out_YT, torch.float32, "out_YT"),
        _ptr(out_grid, torch.float32, "out_grid"), _ptr(out_mean, torch.float64, "out_mean"),
        _ptr(out_var, torch.float64, "out_var"), _ptr(ws), ws.numel(), _stream(stream)))
    return ws


def cdcq_inverse(zn, y, out=None, stream=None):
    """G^{-1} of the quantile-coordinate 7L-CDC scheme (see include/sevenleague.h): zn FP32
    [n_maps, m] marginal nodes, y FP64 [n_maps, n_y]; returns FP64 [n_maps, n_y]."""
    torch = _torch()
    L = load()
    n_maps, m = zn.shape
    n_y = y.shape[1]
    if out is None:
        out = torch.empty((n_maps, n_y), dtype=torch.float64, device=zn.device)
    _check(L.sl_cdcq_inverse(m, _ptr(zn, torch.float32, "zn"), n_maps, _ptr(y, torch.float64, "y"), n_y,
                             _ptr(out, torch.float64, "out"), _stream(stream)))
    return out


def cdc_tables(ws, n_sets, n_steps):
    """View of the tables a 7L-CDC call left in its workspace: FP32 [n_sets, n_steps, 224]."""
    n = n_sets * n_steps * CDC_TABLE_FLOATS
    return ws[256:256 + 4 * n].view(_torch().float32).view(n_sets, n_steps, CDC_TABLE_FLOATS)


def adjoint_workspace_size(total_paths, n_sets, n_steps, ckpt_k, p):
    return int(load().sl_adjoint_workspace_size(total_paths, n_sets, n_steps, ckpt_k, p))


def seven_league_adjoint(model, net, theta, Y0, path_offsets, T, n_steps, m, seed, K, ckpt_k=8,
                         seed_grad=None, out_paths=None, total_paths=None, ws=None, stream=None):
    """Returns (value [n_sets], dY0 [n_sets], dtheta [n_sets, p]) as FP64 device tensors."""
    torch = _torch()
    L = load()
    n_sets = path_offsets.numel() - 1
    p = theta.shape[1] if theta.dim() == 2 else theta.numel() // max(n_sets, 1)
    if total_paths is None:
        total_paths = int(path_offsets[-1].item())
    dev = theta.device
    value = torch.empty(n_sets, dtype=torch.float64, device=dev)
    dY0 = torch.empty(n_sets, dtype=torch.float64, device=dev)
    dth = torch.empty((n_sets, p), dtype=torch.float64, device=dev)
    if ws is None:
        ws = _workspace(L.sl_adjoint_workspace_size(total_paths, n_sets, n_steps, ckpt_k, p), dev)
    netp = ctypes.byref(net) if net is not None else None
    _check(L.seven_league_adjoint(
        model, netp, _ptr(theta, torch.float32, "theta"), p, _ptr(Y0, torch.float32, "Y0"),
        _ptr(path_offsets, torch.int64, "path_offsets"), n_sets, int(total_paths), float(T), n_steps, m,
        seed, PAYOFF_CALL, float(K), ckpt_k, _ptr(value), _ptr(dY0), _ptr(dth),
        _ptr(seed_grad, torch.float64, "seed_grad"), _ptr(out_paths, torch.float32, "out_paths"),
        _ptr(ws), ws.numel(), _stream(stream)))
    return value, dY0, dth


class SevenLeagueCall:
    """torch.autograd.Function: E[max(Y_T - K, 0)] per set as a differentiable
    function of (Y0, theta); forward and backward both run the adjoint kernel
    (the backward passes the upstream gradient in as seed_grad)."""

    @staticmethod
    def apply(Y0, theta, **kw):
        return _autograd_fn().apply(Y0, theta, kw)


_FN = None


def _autograd_fn():
    global _FN
    if _FN is None:
        torch = _torch()

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, Y0, theta, kw):
                ctx.kw = kw
                ctx.save_for_backward(Y0, theta)
                v, _, _ = seven_league_adjoint(kw["model"], kw.get("net"), theta.detach().float().contiguous(),
                                               Y0.detach().float().contiguous(), kw["path_offsets"], kw["T"],
                                               kw["n_steps"], kw["m"], kw["seed"], kw["K"], kw.get("ckpt_k", 8))
                return v

            @staticmethod
            def backward(ctx, gv):
                Y0, theta = ctx.saved_tensors
                kw = ctx.kw
                _, d0, dth = seven_league_adjoint(kw["model"], kw.get("net"), theta.detach().float().contiguous(),
                                                  Y0.detach().float().contiguous(), kw["path_offsets"], kw["T"],
                                                  kw["n_steps"], kw["m"], kw["seed"], kw["K"], kw.get("ckpt_k", 8),
                                                  seed_grad=gv.detach().double().contiguous())
                return d0.to(Y0.dtype), dth.to(theta.dtype), None

        _FN = _Fn
    return _FN


# ---------------------------------------------------------------------------
# Offline stage
# ---------------------------------------------------------------------------
def em_terminal(sde, theta, Yi, dt, n_paths, n_fine, seed, out=None, stream=None):
    torch = _torch()
    L = load()
    n_rows = Yi.numel()
    if out is None:
        out = torch.empty((n_rows, n_paths), dtype=torch.float32, device=Yi.device)
    _check(L.sl_em_terminal(sde, _ptr(theta, torch.float32, "theta"), _ptr(Yi, torch.float32, "Yi"),
                            _ptr(dt, torch.float32, "dt"), n_rows, int(n_paths), n_fine, seed,
                            _ptr(out, torch.float32, "out"), _stream(stream)))
    return out


def segmented_select(values, seg_offsets, ranks, out=None, ws=None, stream=None):
    torch = _torch()
    L = load()
    n_seg = seg_offsets.numel() - 1
    r = np.ascontiguousarray(np.asarray(ranks, dtype=np.int64))
    if out is None:
        out = torch.empty((n_seg, r.size), dtype=torch.float32, device=values.device)
    if ws is None:
        ws = _workspace(L.sl_select_workspace_size(n_seg, r.size), values.device)
    _check(L.sl_segmented_select(_ptr(values, torch.float32, "values"),
                                 _ptr(seg_offsets, torch.int64, "seg_offsets"), n_seg,
                                 r.ctypes.data, r.size, _ptr(out, torch.float32, "out"), _ptr(ws),
                                 ws.numel(), _stream(stream)))
    return out


def em_labels_workspace_size(n_rows, n_paths, m):
    return int(load().sl_em_labels_workspace_size(n_rows, n_paths, m))


def em_collocation_labels(sde, theta, Yi, dt, n_paths, n_fine, m, seed, labels=None, ws=None,
                          stream=None):
    torch = _torch()
    L = load()
    n_rows = Yi.numel()
    if labels is None:
        labels = torch.empty((n_rows, m), dtype=torch.float32, device=Yi.device)
    if ws is None:
        ws = _workspace(L.sl_em_labels_workspace_size(n_rows, n_paths, m), Yi.device)
    _check(L.em_collocation_labels(sde, _ptr(theta, torch.float32, "theta"),
                                   _ptr(Yi, torch.float32, "Yi"), _ptr(dt, torch.float32, "dt"),
                                   n_rows, int(n_paths), n_fine, m, seed,
                                   _ptr(labels, torch.float32, "labels"), _ptr(ws), ws.numel(),
                                   _stream(stream)))
    return labels


def em_collocation_labels_noalloc(sde, theta, Yi, dt, n_paths, n_fine, m, seed, labels=None, stream=None):
    """em_collocation_labels without a caller workspace (the library's fixed
    device buffer; see include/sevenleague.h for its limit and its rules)."""
    torch = _torch()
    L = load()
    n_rows = Yi.numel()
    if labels is None:
        labels = torch.empty((n_rows, m), dtype=torch.float32, device=Yi.device)
    _check(L.em_collocation_labels_noalloc(sde, _ptr(theta, torch.float32, "theta"), _ptr(Yi, torch.float32, "Yi"),
                                           _ptr(dt, torch.float32, "dt"), n_rows, int(n_paths), n_fine, m, seed,
                                           _ptr(labels, torch.float32, "labels"), _stream(stream)))
    return labels


def em_labels_noalloc_max_samples():
    return int(load().sl_em_labels_noalloc_max_samples())


# ---------------------------------------------------------------------------
# Training of the network
# ---------------------------------------------------------------------------
def train_workspace_size(d_in, m, batch):
    return int(load().sl_train_workspace_size(d_in, m, batch))


def mlp_forward(net, feats, out=None, stream=None):
    torch = _torch()
    L = load()
    n = feats.shape[0]
    if out is None:
        out = torch.empty((n, net.m), dtype=torch.float32, device=feats.device)
    _check(L.sl_mlp_forward(ctypes.byref(net), _ptr(feats, torch.float32, "feats"), n,
                            _ptr(out, torch.float32, "out"), _stream(stream)))
    return out


def mse_grad(net, feats, labels, rows=None, stream=None):
    """(loss tensor [1], grad tensor [n_params]) of the MSE over the given rows."""
    torch = _torch()
    L = load()
    n = feats.shape[0] if rows is None else rows.numel()
    grad = torch.empty(n_params(net.d_in, net.m), dtype=torch.float32, device=feats.device)
    loss = torch.empty(1, dtype=torch.float32, device=feats.device)
    ws = _workspace(L.sl_train_workspace_size(net.d_in, net.m, n), feats.device)
    _check(L.sl_mse_grad(ctypes.byref(net), _ptr(feats, torch.float32, "feats"),
                         _ptr(labels, torch.float32, "labels"), _ptr(rows, torch.int32, "rows"), n,
                         _ptr(grad), _ptr(loss), _ptr(ws), ws.numel(), _stream(stream)))
    return loss, grad


def adam_step(params, adam_m, adam_v, grad, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    torch = _torch()
    _check(load().sl_adam_step(_ptr(params, torch.float32), _ptr(adam_m, torch.float32),
                               _ptr(adam_v, torch.float32), _ptr(grad, torch.float32), params.numel(),
                               int(t), lr, b1, b2, eps, _stream(stream)))


def train(params, d_in, m, adam_m, adam_v, t0, feats, labels, batch_rows, batch, lr=1e-3, b1=0.9,
          b2=0.999, eps=1e-8, act=ACT_RELU, losses=None, ws=None, stream=None, prec=PREC_FP32):
    """len(batch_rows)//batch Adam steps in place; returns the per-step losses (device).
    prec=PREC_BF16 trains the BF16-rounded network (see include/sevenleague.h)."""
    torch = _torch()
    L = load()
    nb = batch_rows.numel() // batch
    if losses is None:
        losses = torch.empty(nb, dtype=torch.float32, device=params.device)
    if ws is None:
        ws = _workspace(L.sl_train_workspace_size(d_in, m, batch), params.device)
    _check(L.sl_train(_ptr(params, torch.float32, "params"), d_in, m, act, prec, _ptr(adam_m, torch.float32),
                      _ptr(adam_v, torch.float32), int(t0), _ptr(feats, torch.float32, "feats"),
                      _ptr(labels, torch.float32, "labels"), _ptr(batch_rows, torch.int32, "batch_rows"),
                      nb, batch, lr, b1, b2, eps, _ptr(losses, torch.float32), _ptr(ws), ws.numel(),
                      _stream(stream)))
    return losses
