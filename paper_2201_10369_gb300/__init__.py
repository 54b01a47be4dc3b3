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
WINO_F32, WINO_BF16_TC, WINO_FP16_TC, WINO_SPLIT_BF16X3 = 0, 1, 2, 3
DTYPES = {"f32": WINO_F32, "bf16": WINO_BF16_TC, "fp16": WINO_FP16_TC,
          "split_bf16x3": WINO_SPLIT_BF16X3}
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


class WinoInstance(ctypes.Structure):
    """One planned-sweep instance: size index, subset mask, parameter c."""
    _fields_ = [("size", ctypes.c_int), ("mask", ctypes.c_ubyte), ("c", ctypes.c_double)]


WINO_SWEEP_AUTO, WINO_SWEEP_PERSISTENT, WINO_SWEEP_PERSISTENT3, WINO_SWEEP_PER_SIZE = 0, 1, 2, 3

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
    L.wino_profile_enable.argtypes = [_i]
    L.wino_profile_enable.restype = _i
    L.wino_profile_read.argtypes = [ctypes.c_char_p, _DP, ctypes.POINTER(ctypes.c_int)]
    L.wino_profile_read.restype = _i
    L.wino_kernel_launches.restype = ctypes.c_ulonglong
    L.wino_kernel_launches.argtypes = []
    L.wino_last_error.restype = ctypes.c_char_p
    L.wino_device_ok.restype = _i
    L.wino_shutdown.restype = None
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
    return t.data_ptr()


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
    L = load()
    N, C, H, W = x.shape
    K = w.shape[0]
    pts = _points(points)
    _check(L.wino_conv2d(_ptr(x), _ptr(w), _ptr(y), N, C, K, H, W, pad, pts.ctypes.data_as(_DP),
                         m, r, _dtype(dtype), _stream(stream)))
    return y


def wino_conv1d(x, w, y, points, m: int, r: int, pad: int = 1, dtype="f32", stream=None):
    """y[N][K][Lo] <- Winograd F(m, r) correlation of x[N][C][L] with w[K][C][r]."""
    L = load()
    N, C, Ln = x.shape
    K = w.shape[0]
    pts = _points(points)
    _check(L.wino_conv1d(_ptr(x), _ptr(w), _ptr(y), N, C, K, Ln, pad, pts.ctypes.data_as(_DP),
                         m, r, _dtype(dtype), _stream(stream)))
    return y


def wino_conv2d_f32_noalloc(x, w, y, points, m: int, r: int, pad: int = 1, stream=None):
    """wino_conv2d (FP32) without any device allocation: for callers that
    cannot allocate (inside graph capture, under a framework that owns the
    memory pool).  Uses the library's fixed 16 MiB scratch array; see
    include/wino.h for the limits and the rule that overlapping calls race."""
    L = load()
    N, C, H, W = x.shape
    K = w.shape[0]
    pts = _points(points)
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
    L = load()
    if x.dim() == 3:
        N, C, W = x.shape
        H, dim, r = 1, 1, w.shape[2]
    else:
        N, C, H, W = x.shape
        dim, r = 2, w.shape[3]
    K = w.shape[0]
    _check(L.wino_direct_conv_f64(_ptr(x), _ptr(w), _ptr(y64), dim, N, C, K, H, W, pad, r,
                                  _stream(stream)))
    return y64


def wino_error_stats(yhat, y64, stream=None):
    """(sum|yhat-y|, sum|y|, max|yhat-y|, max|y|) reduced on the device."""
    L = load()
    out = np.zeros(4)
    _check(L.wino_error_stats(_ptr(yhat), _ptr(y64), yhat.numel(), out.ctypes.data_as(_DP),
                              _stream(stream)))
    return tuple(float(v) for v in out)


def wino_error_sweep(c_grid, sizes, subsets, trials: int, seed: int = 0, stream=None):
    """err[n_sizes][n_subsets][n_c] (host FP64); sizes = [(dim, m, r, d)]."""
    L = load()
    cg = np.ascontiguousarray(c_grid, dtype=np.float64)
    sz = (WinoSize * len(sizes))(*[WinoSize(int(a), int(b), int(c), float(d))
                                   for a, b, c, d in sizes])
    mk = np.ascontiguousarray(subsets, dtype=np.uint8)
    err = np.empty((len(sizes), mk.size, cg.size))
    _check(L.wino_error_sweep(cg.ctypes.data_as(_DP), cg.size, sz, len(sizes),
                              mk.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), mk.size, trials,
                              seed, err.ctypes.data_as(_DP), _stream(stream)))
    return err


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
        n = len(instances)
        arr = (WinoInstance * n)()
        for i, (s, mk, c) in enumerate(instances):
            arr[i].size, arr[i].mask, arr[i].c = int(s), int(mk), float(c)
        h = ctypes.c_void_p()
        _check(L.wino_sweep_plan_create(sz, len(sizes), arr, n, trials, seed, mode,
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


def wino_shutdown():
    load().wino_shutdown()
