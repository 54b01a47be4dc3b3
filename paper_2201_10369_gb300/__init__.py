"""Python binding of the GB300 Winograd point-selection library (libwino.so).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels behind the C ABI declared in ``include/wino.h``.  Functions keep
the ABI's names.  Device arrays are torch CUDA tensors (contiguous); the call
is enqueued on ``torch.cuda.current_stream()`` unless a stream is given.
There is no CPU fallback: if libwino.so is missing or no sm_103 device is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

WINO_OK, WINO_EINVAL, WINO_ESINGULAR, WINO_ENOMEM = 0, -1, -2, -3
WINO_ECUDA, WINO_ETIMEOUT, WINO_EUNSUPPORTED = -4, -5, -6
WINO_F32, WINO_BF16_TC, WINO_FP16_TC, WINO_SPLIT_BF16X3, WINO_SPLIT_BF16X6 = 0, 1, 2, 3, 4
DTYPES = {"f32": WINO_F32, "bf16": WINO_BF16_TC, "fp16": WINO_FP16_TC,
          "split_bf16x3": WINO_SPLIT_BF16X3, "split_bf16x6": WINO_SPLIT_BF16X6}
_STATUS = {0: "WINO_OK", -1: "WINO_EINVAL", -2: "WINO_ESINGULAR", -3: "WINO_ENOMEM",
           -4: "WINO_ECUDA", -5: "WINO_ETIMEOUT", -6: "WINO_EUNSUPPORTED"}


class WinoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class WinoSize(ctypes.Structure):
    """One sweep problem size: dim (1 or 2), m, r and the fixed d of Eq. (22)."""
    _fields_ = [("dim", ctypes.c_int), ("m", ctypes.c_int), ("r", ctypes.c_int),
                ("d", ctypes.c_double)]


class WinoPatternCand(ctypes.Structure):
    """One candidate subset of a subset-pattern query (Sec. 6.2)."""
    _fields_ = [("mask", ctypes.c_ubyte), ("best_k", ctypes.c_int), ("best_c", ctypes.c_double),
                ("best_err", ctypes.c_double), ("win_frac", ctypes.c_double)]


class WinoGuidedParams(ctypes.Structure):
    _fields_ = [("top", ctypes.c_int), ("probe", ctypes.c_int), ("refine", ctypes.c_int),
                ("guard", ctypes.c_double)]


class WinoGuidedStats(ctypes.Structure):
    _fields_ = [("evaluated", ctypes.c_int64), ("rows", ctypes.c_int),
                ("fallback_rows", ctypes.c_int), ("phase_ms", ctypes.c_double * 4)]


class WinoInstance(ctypes.Structure):
    """One planned-sweep instance: size index, subset mask, parameter c."""
    _fields_ = [("size", ctypes.c_int), ("mask", ctypes.c_ubyte), ("c", ctypes.c_double)]


WINO_SWEEP_AUTO, WINO_SWEEP_PERSISTENT, WINO_SWEEP_PERSISTENT3, WINO_SWEEP_PER_SIZE = 0, 1, 2, 3
WINO_ORDER_FMA, WINO_ORDER_HUFFMAN, WINO_ORDER_HUFFMAN_MIXED = 0, 1, 2
ORDERS = {"fma": WINO_ORDER_FMA, "huffman": WINO_ORDER_HUFFMAN,
          "huffman_mixed": WINO_ORDER_HUFFMAN_MIXED}

_lib = None
_lock = threading.Lock()
_i, _d, _vp, _sz = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_DP = ctypes.POINTER(ctypes.c_double)


def _declare(L):
    L.wino_make_matrices.argtypes = [_DP, _i, _i, _DP, _DP, _DP]
    L.wino_conv1d.argtypes = [_vp, _vp, _vp] + [_i] * 5 + [_DP, _i, _i, _i, _vp]
    L.wino_conv2d.argtypes = [_vp, _vp, _vp] + [_i] * 6 + [_DP, _i, _i, _i, _vp]
    L.wino_workspace_bytes.argtypes = [_i] * 8
    L.wino_workspace_bytes.restype = _sz
    L.wino_set_workspace.argtypes = [_vp, _sz]
    L.wino_direct_conv_f64.argtypes = [_vp, _vp, _vp] + [_i] * 8 + [_vp]
    L.wino_error_stats.argtypes = [_vp, _vp, ctypes.c_int64, _DP, _vp]
    L.wino_error_sweep.argtypes = [_DP, _i, ctypes.POINTER(WinoSize), _i,
                                   ctypes.POINTER(ctypes.c_ubyte), _i, _i, ctypes.c_ulonglong,
                                   _DP, _vp]
    L.wino_instance_matrices.argtypes = [_DP, _i, WinoSize, ctypes.c_uint, _DP, _DP, _DP,
                                         ctypes.POINTER(ctypes.c_ubyte), _vp]
    L.wino_instance_matrices.restype = _i
    L.wino_conv2d_f32_noalloc.argtypes = [_vp, _vp, _vp] + [_i] * 6 + [_DP, _i, _i, _vp]
    L.wino_conv2d_f32_noalloc.restype = _i
    L.wino_sweep_plan_create.argtypes = [ctypes.POINTER(WinoSize), _i,
                                         ctypes.POINTER(WinoInstance), ctypes.c_int64, _i,
                                         ctypes.c_ulonglong, _i, ctypes.POINTER(_vp)]
    L.wino_sweep_plan_create.restype = _i
    L.wino_sweep_plan_set_deadline.argtypes = [_vp, _d]
    L.wino_sweep_plan_set_deadline.restype = _i
    L.wino_sweep_plan_run.argtypes = [_vp, _DP, _vp]
    L.wino_sweep_plan_run.restype = _i
    L.wino_sweep_plan_info.argtypes = [_vp] + [ctypes.POINTER(_i)] * 3
    L.wino_sweep_plan_info.restype = _i
    L.wino_sweep_plan_destroy.argtypes = [_vp]
    L.wino_sweep_plan_destroy.restype = None
    _FP = ctypes.POINTER(ctypes.c_float)
    L.wino_mlp_create.argtypes = [ctypes.c_ulonglong, ctypes.POINTER(_vp)]
    L.wino_mlp_set_params.argtypes = [_vp, _FP]
    L.wino_mlp_get_params.argtypes = [_vp, _FP, _i]
    L.wino_mlp_features.argtypes = [ctypes.POINTER(WinoSize), _i, ctypes.POINTER(WinoInstance),
                                    ctypes.c_int64, _vp, _vp]
    L.wino_mlp_loss_grad.argtypes = [_vp, _vp, _vp, _i, _FP, _DP, _vp]
    L.wino_mlp_train.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _i, _i, ctypes.c_float, _vp]
    L.wino_mlp_predict.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp]
    L.wino_topk_rows.argtypes = [_vp, _i, _i, _i, _vp, _vp]
    L.wino_mlp_grid_features.argtypes = [ctypes.POINTER(WinoSize), _i, ctypes.POINTER(_i),
                                         ctypes.POINTER(ctypes.c_ubyte), _i, _DP, _i, _vp, _vp]
    L.wino_mlp_grid_features.restype = _i
    L.wino_sweep_plan_set_c.argtypes = [_vp, _DP, ctypes.c_int64]
    L.wino_sweep_plan_set_c.restype = _i
    for nm in ("wino_mlp_create", "wino_mlp_set_params", "wino_mlp_get_params",
               "wino_mlp_features", "wino_mlp_loss_grad", "wino_mlp_train", "wino_mlp_predict",
               "wino_topk_rows"):
        getattr(L, nm).restype = _i
    L.wino_mlp_destroy.argtypes = [_vp]
    L.wino_mlp_destroy.restype = None
    L.wino_profile_enable.argtypes = [_i]
    L.wino_profile_enable.restype = _i
    L.wino_profile_read.argtypes = [ctypes.c_char_p, _DP, ctypes.POINTER(ctypes.c_int)]
    L.wino_profile_read.restype = _i
    L.wino_kernel_launches.restype = ctypes.c_ulonglong
    L.wino_kernel_launches.argtypes = []
    L.wino_last_error.restype = ctypes.c_char_p
    L.wino_device_ok.restype = _i
    L.wino_pointset_error.argtypes = [_i, _i, _i, _DP, _i, _i, ctypes.c_ulonglong, _DP, _vp]
    L.wino_pointset_error.restype = _i
    L.wino_pointset_error_order.argtypes = [_i, _i, _i, _DP, _i, _i, ctypes.c_ulonglong, _i, _DP,
                                            _vp]
    L.wino_pointset_error_order.restype = _i
    L.wino_error_sweep_order.argtypes = [_DP, _i, ctypes.POINTER(WinoSize), _i,
                                         ctypes.POINTER(ctypes.c_ubyte), _i, _i,
                                         ctypes.c_ulonglong, _i, _DP, _vp]
    L.wino_error_sweep_order.restype = _i
    L.wino_pointset_error_kron.argtypes = [_i, _i, _DP, _i, _i, ctypes.c_ulonglong, _i, _DP,
                                           _vp]
    L.wino_pointset_error_kron.restype = _i
    L.wino_wait_error.argtypes = [ctypes.POINTER(ctypes.c_int)]
    L.wino_wait_error.restype = _i
    L.wino_wait_probe.argtypes = [_i, ctypes.POINTER(ctypes.c_longlong), ctypes.c_void_p]
    L.wino_wait_probe.restype = _i
    L.wino_shutdown.restype = None
    L.wino_subset_pattern.argtypes = [_DP, ctypes.POINTER(ctypes.c_ubyte), _i, _DP, _i, WinoSize,
                                      ctypes.c_ubyte, _d, _d, ctypes.POINTER(WinoPatternCand), _i,
                                      ctypes.POINTER(_i)]
    L.wino_subset_pattern.restype = _i
    _UB = ctypes.POINTER(ctypes.c_ubyte)
    L.wino_guided_create.argtypes = [_vp, ctypes.POINTER(WinoSize), _i, _UB, _i, _DP, _i, _i,
                                     ctypes.c_ulonglong, ctypes.POINTER(WinoGuidedParams),
                                     ctypes.POINTER(_vp)]
    L.wino_guided_create.restype = _i
    L.wino_guided_run.argtypes = [_vp, _DP, _DP, ctypes.POINTER(WinoGuidedStats), _vp]
    L.wino_guided_run.restype = _i
    L.wino_guided_destroy.argtypes = [_vp]
    L.wino_guided_destroy.restype = None
    L.wino_random_search.argtypes = [ctypes.POINTER(WinoSize), _i, _UB, _i, _DP, _i, _i, _i,
                                     ctypes.c_ulonglong, _DP, _vp]
    L.wino_random_search.restype = _i
    L.wino_cd_sweep.argtypes = [_i, _i, _i, _DP, _i, _DP, _i, _UB, _i, _i, ctypes.c_ulonglong,
                                _DP, _vp]
    L.wino_cd_sweep.restype = _i
    L.wino_pipe_peak.argtypes = [_i, _i, _i, _DP, _DP, _vp]
    L.wino_pipe_peak.restype = _i
    for name in ("wino_make_matrices", "wino_conv1d", "wino_conv2d", "wino_set_workspace",
                 "wino_direct_conv_f64", "wino_error_stats", "wino_error_sweep"):
        getattr(L, name).restype = _i
    _declare_more(L)


def _declare_more(L):
    """Entry points added by later modules of the library (see below)."""
    for fn in _EXTRA_DECLS:
        fn(L)


_EXTRA_DECLS = []


def load(path: str | None = None):
    """Loads libwino.so (built in-tree by ``build()``); raises if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            so = path or _build.SO
            if not os.path.exists(so):
                raise RuntimeError("libwino.so not built (%s); run paper_2201_10369_gb300.build()"
                                   % so)
            L = ctypes.CDLL(so)
            _declare(L)
            _lib = L
    return _lib


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the CUDA library for sm_103a in-tree and returns its path."""
    return _build.build(force=force, verbose=verbose)


def lib_path() -> str:
    return _build.SO


def _check(st: int):
    if st != WINO_OK:
        msg = _lib.wino_last_error().decode(errors="replace") if _lib else ""
        raise WinoError(st, msg)


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    import torch
    if t.device.index != torch.cuda.current_device():
        raise ValueError("tensor on cuda:%s, but the current device is cuda:%d"
                         % (t.device.index, torch.cuda.current_device()))
    return t.data_ptr()


def _want(name, t, dtype, shape=None, ndim=None):
    """Checks a tensor argument's dtype and shape before any ABI call (the
    library indexes device memory from the sizes alone, so a wrong dtype or
    an undersized tensor would be read or written out of bounds)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s must be a torch tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if ndim is not None and t.dim() != ndim:
        raise ValueError("%s must have %d dimensions, got shape %s" % (name, ndim, tuple(t.shape)))
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))


def _check_layer(x, w, y, pts, m, r, pad, dim):
    """Validates the arguments of a layer call (x, w, y FP32; shapes
    x [N][C](H)[W], w [K][C](r)[r], y [N][K](Ho)[Wo]; m + r - 1 points)."""
    import torch
    if m < 1 or r < 1 or pad < 0:
        raise ValueError("need m >= 1, r >= 1, pad >= 0")
    if pts.ndim != 1 or pts.size != m + r - 1:
        raise ValueError("need alpha = m + r - 1 = %d points, got %d" % (m + r - 1, pts.size))
    _want("x", x, torch.float32, ndim=dim + 2)
    N, C = x.shape[0], x.shape[1]
    sp = tuple(x.shape[2:])
    _want("w", w, torch.float32, ndim=dim + 2)
    K = w.shape[0]
    _want("w", w, torch.float32, shape=(K, C) + (r,) * dim)
    out = tuple(v + 2 * pad - r + 1 for v in sp)
    if min(out) < 1:
        raise ValueError("kernel larger than the padded input")
    _want("y", y, torch.float32, shape=(N, K) + out)


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _points(points) -> np.ndarray:
    return np.ascontiguousarray(points, dtype=np.float64)


# ---------------------------------------------------------------------------
# ABI calls
# ---------------------------------------------------------------------------

def wino_make_matrices(points, m: int, r: int):
    """FP64 (AT[m][alpha], G[alpha][r], BT[alpha][alpha]), canonical order."""
    L = load()
    a = m + r - 1
    pts = _points(points)
    if pts.size != a:
        raise ValueError("need alpha = m + r - 1 points")
    AT, G, BT = np.zeros((m, a)), np.zeros((a, r)), np.zeros((a, a))
    _check(L.wino_make_matrices(pts.ctypes.data_as(_DP), m, r, AT.ctypes.data_as(_DP),
                                G.ctypes.data_as(_DP), BT.ctypes.data_as(_DP)))
    return AT, G, BT


def _dtype(dtype) -> int:
    return DTYPES[dtype] if isinstance(dtype, str) else int(dtype)


def wino_conv2d(x, w, y, points, m: int, r: int, pad: int = 1, dtype="f32", stream=None):
    """y[N][K][Ho][Wo] <- Winograd F(m x m, r x r) correlation of x with w."""
    pts = _points(points)
    _check_layer(x, w, y, pts, m, r, pad, 2)
    L = load()
    N, C, H, W = x.shape
    K = w.shape[0]
    _check(L.wino_conv2d(_ptr(x), _ptr(w), _ptr(y), N, C, K, H, W, pad, pts.ctypes.data_as(_DP),
                         m, r, _dtype(dtype), _stream(stream)))
    return y


def wino_conv1d(x, w, y, points, m: int, r: int, pad: int = 1, dtype="f32", stream=None):
    """y[N][K][Lo] <- Winograd F(m, r) correlation of x[N][C][L] with w[K][C][r]."""
    pts = _points(points)
    _check_layer(x, w, y, pts, m, r, pad, 1)
    L = load()
    N, C, Ln = x.shape
    K = w.shape[0]
    _check(L.wino_conv1d(_ptr(x), _ptr(w), _ptr(y), N, C, K, Ln, pad, pts.ctypes.data_as(_DP),
                         m, r, _dtype(dtype), _stream(stream)))
    return y


def wino_conv2d_f32_noalloc(x, w, y, points, m: int, r: int, pad: int = 1, stream=None):
    """wino_conv2d (FP32) without any device allocation: for callers that
    cannot allocate (inside graph capture, under a framework that owns the
    memory pool).  Uses the library's fixed 16 MiB scratch array; see
    include/wino.h for the limits and the rule that overlapping calls race."""
    pts = _points(points)
    _check_layer(x, w, y, pts, m, r, pad, 2)
    L = load()
    N, C, H, W = x.shape
    K = w.shape[0]
    _check(L.wino_conv2d_f32_noalloc(_ptr(x), _ptr(w), _ptr(y), N, C, K, H, W, pad,
                                     pts.ctypes.data_as(_DP), m, r, _stream(stream)))
    return y


def wino_workspace_bytes(N, C, K, H, W, m, r, dtype="f32") -> int:
    return int(load().wino_workspace_bytes(N, C, K, H, W, m, r, _dtype(dtype)))


def wino_set_workspace(buf=None, nbytes: int = 0):
    """Hands the library caller-owned scratch (a CUDA tensor), or reverts to
    internal scratch when called with no buffer."""
    L = load()
    if buf is None:
        _check(L.wino_set_workspace(None, 0))
    else:
        _check(L.wino_set_workspace(_ptr(buf), nbytes or buf.numel() * buf.element_size()))


def wino_direct_conv_f64(x, w, y64, pad: int = 1, stream=None):
    """FP64 direct correlation (Eq. (1)); x, w FP32 CUDA tensors, y64 FP64."""
    import torch
    _want("x", x, torch.float32)
    if x.dim() not in (3, 4):
        raise ValueError("x must be [N][C][W] or [N][C][H][W]")
    dim = x.dim() - 2
    _want("w", w, torch.float32, ndim=x.dim())
    r = w.shape[-1]
    _want("w", w, torch.float32, shape=(w.shape[0], x.shape[1]) + (r,) * dim)
    if pad < 0 or min(v + 2 * pad - r + 1 for v in x.shape[2:]) < 1:
        raise ValueError("need pad >= 0 and a kernel no larger than the padded input")
    _want("y64", y64, torch.float64,
          shape=(x.shape[0], w.shape[0]) + tuple(v + 2 * pad - r + 1 for v in x.shape[2:]))
    L = load()
    if dim == 1:
        N, C, W = x.shape
        H = 1
    else:
        N, C, H, W = x.shape
    K = w.shape[0]
    _check(L.wino_direct_conv_f64(_ptr(x), _ptr(w), _ptr(y64), dim, N, C, K, H, W, pad, r,
                                  _stream(stream)))
    return y64


def wino_error_stats(yhat, y64, stream=None):
    """(sum|yhat-y|, sum|y|, max|yhat-y|, max|y|) reduced on the device."""
    import torch
    _want("yhat", yhat, torch.float32)
    _want("y64", y64, torch.float64)
    if yhat.numel() != y64.numel():
        raise ValueError("yhat and y64 must hold the same number of elements")
    L = load()
    out = np.zeros(4)
    _check(L.wino_error_stats(_ptr(yhat), _ptr(y64), yhat.numel(), out.ctypes.data_as(_DP),
                              _stream(stream)))
    return tuple(float(v) for v in out)


def wino_error_sweep(c_grid, sizes, subsets, trials: int, seed: int = 0, stream=None,
                     order: str = "fma"):
    """err[n_sizes][n_subsets][n_c] (host FP64); sizes = [(dim, m, r, d)].
    ``order``: 'fma' (wino_error_sweep), 'huffman' or 'huffman_mixed'
    (wino_error_sweep_order)."""
    L = load()
    cg = np.ascontiguousarray(c_grid, dtype=np.float64)
    sz = (WinoSize * len(sizes))(*[WinoSize(int(a), int(b), int(c), float(d))
                                   for a, b, c, d in sizes])
    mk = np.ascontiguousarray(subsets, dtype=np.uint8)
    err = np.empty((len(sizes), mk.size, cg.size))
    args = (cg.ctypes.data_as(_DP), cg.size, sz, len(sizes),
            mk.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), mk.size, trials, seed)
    if order == "fma":
        _check(L.wino_error_sweep(*args, err.ctypes.data_as(_DP), _stream(stream)))
    else:
        _check(L.wino_error_sweep_order(*args, ORDERS[order], err.ctypes.data_as(_DP),
                                        _stream(stream)))
    return err


def wino_subset_pattern(err, masks, c_grid, size, base_mask: int, c_lo: float = 1.0,
                        c_hi: float = float("inf")):
    """The subset-pattern query (Sec. 6.2, Tables 2-6) over one size's sweep
    errors err[n_masks][n_c]: the candidate subsets of `base_mask` ranked by
    least error in the c window, as dicts {mask, best_k, best_c, best_err,
    win_frac}; the first is the base's pattern."""
    e = np.ascontiguousarray(err, dtype=np.float64)
    mk = np.ascontiguousarray(masks, dtype=np.uint8)
    cg = np.ascontiguousarray(c_grid, dtype=np.float64)
    if e.shape != (mk.size, cg.size):
        raise ValueError("err must be [n_masks][n_c]")
    dim, m, r, d = size
    out = (WinoPatternCand * 16)()
    n = _i(0)
    _check(load().wino_subset_pattern(e.ctypes.data_as(_DP), mk.ctypes.data_as(ctypes.POINTER(
        ctypes.c_ubyte)), mk.size, cg.ctypes.data_as(_DP), cg.size, WinoSize(dim, m, r, d),
        int(base_mask), float(c_lo), float(c_hi), out, 16, ctypes.byref(n)))
    return [{"mask": int(o.mask), "best_k": int(o.best_k), "best_c": float(o.best_c),
             "best_err": float(o.best_err), "win_frac": float(o.win_frac)}
            for o in out[:min(n.value, 16)]]


def wino_instance_matrices(c_grid, size, mask: int, stream=None):
    """Device-built FP64 matrices of the sweep instances (size, mask, c_k):
    (AT[n][m][alpha], G[n][alpha][r], BT[n][alpha][alpha], singular[n])."""
    L = load()
    cg = np.ascontiguousarray(c_grid, dtype=np.float64)
    dim, m, r, d = size
    a = m + r - 1
    n = cg.size
    AT, G, BT = np.zeros((n, m, a)), np.zeros((n, a, r)), np.zeros((n, a, a))
    sing = np.zeros(n, dtype=np.uint8)
    _check(L.wino_instance_matrices(cg.ctypes.data_as(_DP), n, WinoSize(dim, m, r, d), mask,
                                    AT.ctypes.data_as(_DP), G.ctypes.data_as(_DP),
                                    BT.ctypes.data_as(_DP),
                                    sing.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                    _stream(stream)))
    return AT, G, BT, sing.astype(bool)


class SweepPlan:
    """A planned sweep (wino_sweep_plan_*): build once, run many times.

    ``instances`` is a sequence of (size index, mask, c); ``run()`` returns the
    errors in that order (NaN where the mask is invalid for its size)."""

    def __init__(self, sizes, instances, trials: int, seed: int = 0, mode: int = WINO_SWEEP_AUTO):
        L = load()
        self._L = L
        sz = (WinoSize * len(sizes))(*[WinoSize(int(a), int(b), int(c), float(d))
                                       for a, b, c, d in sizes])
        arr, ptr = _instances(instances)
        n = arr.size
        h = ctypes.c_void_p()
        _check(L.wino_sweep_plan_create(sz, len(sizes), ptr, n, trials, seed, mode,
                                        ctypes.byref(h)))
        self._h = h
        self.n = n

    def set_deadline(self, max_ms: float):
        _check(self._L.wino_sweep_plan_set_deadline(self._h, float(max_ms)))

    def run(self, stream=None) -> np.ndarray:
        err = np.empty(self.n)
        st = 0 if stream is None else _stream(stream)
        _check(self._L.wino_sweep_plan_run(self._h, err.ctypes.data_as(_DP), st or None))
        return err

    def info(self):
        m, g, n = _i(), _i(), _i()
        _check(self._L.wino_sweep_plan_info(self._h, ctypes.byref(m), ctypes.byref(g),
                                            ctypes.byref(n)))
        return {"mode": m.value, "grid": g.value, "items": n.value}

    def close(self):
        if getattr(self, "_h", None):
            self._L.wino_sweep_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_PARAMS = 1153


# numpy layout of wino_instance (int size, unsigned char mask, padding, double c)
INSTANCE_DTYPE = np.dtype([("size", "<i4"), ("mask", "u1"), ("pad", "u1", (3,)), ("c", "<f8")])


def instance_array(size_idx, mask, c) -> np.ndarray:
    """Instances as an INSTANCE_DTYPE array (broadcasting the three fields)."""
    c = np.asarray(c, dtype=np.float64)
    size_idx, mask, c = np.broadcast_arrays(np.asarray(size_idx), np.asarray(mask), c)
    a = np.zeros(c.size, dtype=INSTANCE_DTYPE)
    a["size"] = size_idx.ravel()
    a["mask"] = mask.ravel()
    a["c"] = c.ravel()
    return a


def _instances(instances):
    """(array, ctypes pointer) of wino_instance records from (size, mask, c)
    tuples or an INSTANCE_DTYPE array."""
    if isinstance(instances, np.ndarray) and instances.dtype == INSTANCE_DTYPE:
        a = np.ascontiguousarray(instances)
    else:
        s, m, c = zip(*instances) if len(instances) else ((), (), ())
        a = instance_array(np.array(s, dtype=np.int32), np.array(m, dtype=np.uint8),
                           np.array(c, dtype=np.float64))
    return a, a.ctypes.data_as(ctypes.POINTER(WinoInstance))


def _sizes(sizes):
    return (WinoSize * len(sizes))(*[WinoSize(int(a), int(b), int(c), float(d))
                                     for a, b, c, d in sizes])


class Surrogate:
    """The learned surrogate (wino_mlp_*): a 16-64-1 GELU network on the
    device predicting log10 of an instance's sweep error."""

    def __init__(self, seed: int = 0):
        L = load()
        self._L = L
        h = ctypes.c_void_p()
        _check(L.wino_mlp_create(seed, ctypes.byref(h)))
        self._h = h

    def params(self, working: bool = False) -> np.ndarray:
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(self._L.wino_mlp_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           1 if working else 0))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._L.wino_mlp_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def features(self, sizes, instances, stream=None):
        return instance_features(sizes, instances, stream)

    @staticmethod
    def _check_xy(X, y=None):
        import torch
        _want("X", X, torch.float32, ndim=2)
        if X.shape[1] != 16:
            raise ValueError("X must be [n][16] features")
        if y is not None:
            _want("y", y, torch.float32, shape=(X.shape[0],))

    def loss_grad(self, X, y, stream=None):
        self._check_xy(X, y)
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(self._L.wino_mlp_loss_grad(self._h, _ptr(X), _ptr(y), X.shape[0],
                                          g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          ctypes.byref(loss), _stream(stream)))
        return loss.value, g

    def set_output_bias(self, b: float):
        """Starts the output bias at b (e.g. the label mean); resets Adam."""
        p = self.params()
        p[-1] = b
        self.set_params(p)

    def train(self, X, y, batch: int = 4096, epochs: int = 1, lr: float = 1e-3, stream=None):
        self._check_xy(X, y)
        _check(self._L.wino_mlp_train(self._h, _ptr(X), _ptr(y), X.shape[0], batch, epochs, lr,
                                      _stream(stream)))

    def predict(self, X, stream=None):
        import torch
        self._check_xy(X)
        out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(self._L.wino_mlp_predict(self._h, _ptr(X), X.shape[0], _ptr(out), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._L.wino_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wino_topk_rows(vals, k: int, stream=None):
    """Indices (CUDA int32 [rows][k]) of the k smallest values of each row."""
    import torch
    _want("vals", vals, torch.float32, ndim=2)
    rows, cols = vals.shape
    if not 1 <= k <= cols:
        raise ValueError("need 1 <= k <= cols")
    idx = torch.empty((rows, k), dtype=torch.int32, device=vals.device)
    _check(load().wino_topk_rows(_ptr(vals), rows, cols, k, _ptr(idx), _stream(stream)))
    return idx


def valid_masks(size, masks):
    """The masks of `masks` valid for size (dim, m, r, d): popcount alpha - 2,
    and bits 4 and 7 unused when |d| = 1 (the rule of wino_error_sweep)."""
    dim, m, r, d = size
    out = []
    for mk in masks:
        mk = int(mk)
        if bin(mk).count("1") != m + r - 3:
            continue
        if abs(d) == 1.0 and (mk & 0x90):
            continue
        out.append(mk)
    return out


LABEL_CLIP = -3.0  # labels are min(log10 err, -3)


def instance_features(sizes, instances, stream=None):
    """Surrogate features (device [n][16]) of instances (tuples or an
    INSTANCE_DTYPE array)."""
    import torch
    arr, ptr = _instances(instances)
    X = torch.empty((arr.size, 16), dtype=torch.float32, device="cuda")
    _check(load().wino_mlp_features(_sizes(sizes), len(sizes), ptr, arr.size, _ptr(X),
                                    _stream(stream)))
    return X


def surrogate_training_set(sizes, masks, n: int, trials: int, seed: int = 0, c_lo=0.05, c_hi=20.0):
    """n random instances (size, valid mask, c log-uniform in [c_lo, c_hi]),
    their sweep errors from one planned launch, and labels min(log10 err,
    LABEL_CLIP); instances whose points coincide are dropped.  Returns
    (instances as an INSTANCE_DTYPE array, X, y) with X, y on the device."""
    import torch
    rng = np.random.default_rng(seed)
    per = [np.array(valid_masks(s, masks), dtype=np.uint8) for s in sizes]
    cand = np.array([i for i, p in enumerate(per) if p.size], dtype=np.int32)
    sidx = cand[rng.integers(cand.size, size=n)]
    mk = np.empty(n, dtype=np.uint8)
    for s in cand:
        sel = sidx == s
        mk[sel] = per[s][rng.integers(per[s].size, size=int(sel.sum()))]
    c = np.exp(rng.uniform(np.log(c_lo), np.log(c_hi), n))
    inst = instance_array(sidx, mk, c)
    plan = SweepPlan(sizes, inst, trials, seed=seed, mode=WINO_SWEEP_PERSISTENT)
    try:
        err = plan.run()
    finally:
        plan.close()
    keep = np.isfinite(err) & (err > 0)
    inst = inst[keep]
    # errors above 1e-3 are far from any useful point set; clipping them keeps
    # the rare near-singular spikes from dominating the squared loss
    y = torch.from_numpy(np.minimum(np.log10(err[keep]), LABEL_CLIP).astype(np.float32)).cuda()
    return inst, instance_features(sizes, inst), y


class GuidedSearch:
    """Surrogate-guided search of a c grid for every valid (size, mask) row
    (wino_guided_create / wino_guided_run; the method is described in
    include/wino.h): the network's `top` proposals and `probe` random grid
    points verified in one planned launch, the neighbours of the network's
    best refined in a second, and rows where the network's region loses to
    `guard` x the random probe swept exhaustively."""

    def __init__(self, model, sizes, masks, c_grid, trials: int, seed: int = 0, top: int = 64,
                 probe: int = 64, refine: int = 32, guard: float = 1.01):
        L = load()
        self._L = L
        self.model, self.sizes = model, list(sizes)
        self.cg = np.ascontiguousarray(c_grid, dtype=np.float64)
        self.masks = np.ascontiguousarray([int(mk) for mk in masks], dtype=np.uint8)
        prm = WinoGuidedParams(int(top), int(probe), int(refine), float(guard))
        h = ctypes.c_void_p()
        _check(L.wino_guided_create(model._h, _sizes(sizes), len(sizes),
                                    self.masks.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                    self.masks.size, self.cg.ctypes.data_as(_DP), self.cg.size,
                                    int(trials), int(seed), ctypes.byref(prm), ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        shape = (len(self.sizes), self.masks.size)
        best, best_c = np.empty(shape), np.empty(shape)
        st = WinoGuidedStats()
        _check(self._L.wino_guided_run(self._h, best.ctypes.data_as(_DP),
                                       best_c.ctypes.data_as(_DP), ctypes.byref(st),
                                       _stream(stream)))
        ph = list(st.phase_ms)
        return {"best_err": best, "best_c": best_c, "evaluated": int(st.evaluated),
                "fallback_rows": int(st.fallback_rows), "rows": int(st.rows),
                "phase_ms": {"rank": ph[0], "verify": ph[1], "refine": ph[2], "fallback": ph[3]}}

    def close(self):
        if getattr(self, "_h", None):
            self._L.wino_guided_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def random_search(sizes, masks, c_grid, trials: int, budget: int, seed: int = 0, stream=None):
    """The search without the network, at a given per-row budget
    (wino_random_search): best_err [n_sizes][n_masks]."""
    cg = np.ascontiguousarray(c_grid, dtype=np.float64)
    mk = np.ascontiguousarray([int(v) for v in masks], dtype=np.uint8)
    best = np.empty((len(sizes), mk.size))
    _check(load().wino_random_search(_sizes(sizes), len(sizes),
                                     mk.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), mk.size,
                                     cg.ctypes.data_as(_DP), cg.size, int(trials), int(budget),
                                     int(seed), best.ctypes.data_as(_DP), _stream(stream)))
    return best


def guided_sweep(model, sizes, masks, c_grid, trials: int, seed: int = 0, top: int = 64,
                 probe: int = 64, refine: int = 32, guard: float = 1.01):
    """One surrogate-guided search (GuidedSearch built, run once, closed)."""
    gs = GuidedSearch(model, sizes, masks, c_grid, trials, seed, top, probe, refine, guard)
    try:
        return gs.run()
    finally:
        gs.close()


def wino_pointset_error(size, point_sets, trials: int, seed: int = 0, stream=None,
                        order: str = "fma") -> np.ndarray:
    """The sweep metric of explicit point sets on the sweep's trials of size
    (dim, m, r[, d]): each set m + r - 1 values with one +inf, any order.
    ``order`` as for wino_error_sweep."""
    dim, m, r = size[0], size[1], size[2]
    pts = np.ascontiguousarray(point_sets, dtype=np.float64)
    if pts.ndim != 2 or pts.shape[1] != m + r - 1:
        raise ValueError("each point set needs m + r - 1 values")
    err = np.empty(pts.shape[0])
    L = load()
    args = (dim, m, r, pts.ctypes.data_as(_DP), pts.shape[0], trials, seed)
    if order == "fma":
        _check(L.wino_pointset_error(*args, err.ctypes.data_as(_DP), _stream(stream)))
    else:
        _check(L.wino_pointset_error_order(*args, ORDERS[order], err.ctypes.data_as(_DP),
                                           _stream(stream)))
    return err


def cd_sweep(dim: int, m: int, c_grid, d_grid, masks, trials: int, seed: int = 0, r: int = 3,
             stream=None) -> np.ndarray:
    """The two-parameter sweep (wino_cd_sweep; Sec. 4: the c-group with a
    subset of the d-group for larger sizes): err[n_d][n_masks][n_c], NaN
    where a mask is invalid for that d."""
    cg = np.ascontiguousarray(c_grid, dtype=np.float64)
    dg = np.ascontiguousarray(d_grid, dtype=np.float64)
    mk = np.ascontiguousarray([int(v) for v in masks], dtype=np.uint8)
    err = np.empty((dg.size, mk.size, cg.size))
    _check(load().wino_cd_sweep(int(dim), int(m), int(r), cg.ctypes.data_as(_DP), cg.size,
                                dg.ctypes.data_as(_DP), dg.size,
                                mk.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), mk.size,
                                int(trials), int(seed), err.ctypes.data_as(_DP), _stream(stream)))
    return err


def wino_pointset_error_kron(m: int, point_sets, trials: int, seed: int = 0,
                             pairwise: bool = False, r: int = 3, stream=None) -> np.ndarray:
    """The sweep metric of the Kronecker-product form of the 2D tile (Sec. 7)
    for explicit point sets, on the sweep's 2D trials of size (m, r)."""
    pts = np.ascontiguousarray(point_sets, dtype=np.float64)
    if pts.ndim != 2 or pts.shape[1] != m + r - 1:
        raise ValueError("each point set needs m + r - 1 values")
    err = np.empty(pts.shape[0])
    _check(load().wino_pointset_error_kron(m, r, pts.ctypes.data_as(_DP), pts.shape[0], trials,
                                           seed, int(pairwise), err.ctypes.data_as(_DP),
                                           _stream(stream)))
    return err


def grid_instances(sizes, masks, c_grid):
    """All (size, mask, c) of a full grid, in [size][mask][c] order."""
    return [(s, int(mk), float(c)) for s in range(len(sizes)) for mk in masks for c in c_grid]


def wino_kernel_launches() -> int:
    return int(load().wino_kernel_launches())


def wino_profile_enable(on: bool = True):
    _check(load().wino_profile_enable(1 if on else 0))


def wino_profile_read(kernel: str):
    """(total milliseconds, launches) recorded for `kernel` since the last read."""
    L = load()
    ms, n = ctypes.c_double(0.0), ctypes.c_int(0)
    _check(L.wino_profile_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def wino_last_error() -> str:
    return load().wino_last_error().decode(errors="replace")


def wino_device_ok() -> bool:
    return bool(load().wino_device_ok())


def wino_wait_error() -> bool:
    """True when a bounded device wait in a layer kernel gave up on the
    current device since the last call (that layer's output is incomplete);
    clears the flag.  Synchronises the device."""
    f = ctypes.c_int(0)
    _check(load().wino_wait_error(ctypes.byref(f)))
    return bool(f.value)


def wino_wait_probe(polls: int) -> int:
    """Runs the layer kernels' bounded wait on an mbarrier nothing arrives at,
    `polls` polls, on the current stream: the wait gives up and sets the flag
    `wino_wait_error` reports.  Returns the device time of the polls in ns."""
    import torch
    ns = ctypes.c_longlong(0)
    _check(load().wino_wait_probe(int(polls), ctypes.byref(ns),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return int(ns.value)


WINO_PIPE_FP32, WINO_PIPE_FP32X2, WINO_PIPE_FP64 = 0, 1, 2
PIPES = {"fp32": WINO_PIPE_FP32, "fp32x2": WINO_PIPE_FP32X2, "fp64": WINO_PIPE_FP64}


def wino_pipe_peak(kind: str, iters: int, blocks_per_sm: int = 4, stream=None):
    """(TFLOP/s, ms) of one launch of the library's FMA-throughput probe of
    one pipe ('fp32', 'fp32x2' or 'fp64'); synchronises the stream."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().wino_pipe_peak(PIPES[kind], int(iters), int(blocks_per_sm), ctypes.byref(tf),
                                 ctypes.byref(ms), _stream(stream)))
    return tf.value, ms.value


def wino_shutdown():
    load().wino_shutdown()
