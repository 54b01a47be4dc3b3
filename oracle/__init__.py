"""Plain CPU oracle for Winograd point selection -- TEST INFRASTRUCTURE ONLY.

This package is the slow, obviously correct statement of what the GPU library
computes (transform matrices, direct correlation, FP32 Winograd in a fixed
operation order, the error metric and the point sweep, the MLP surrogate's
FP64 forward/backward).  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import it.  It shares no code with
``paper_2201_10369_gb300`` and never imports it.

``build()`` compiles ``wino_oracle.c`` with ``-ffp-contract=off`` into
``oracle/_build/liboracle.so``; the wrappers below are argument marshalling.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "wino_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the C oracle (gcc, no FP contraction).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_SO) >= os.path.getmtime(os.path.join(_HERE, "wino_oracle.h"))):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["cc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Size(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("m", ctypes.c_int), ("r", ctypes.c_int),
                ("d", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            L.orc_make_matrices.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.orc_make_matrices.restype = ctypes.c_int
            L.orc_canonical_points.argtypes = [dp, ctypes.c_int, dp]
            L.orc_direct_f64.argtypes = [fp, fp, dp] + [ctypes.c_int] * 8
            L.orc_direct_f64.restype = None
            for nm in ("orc_tile1d_f32", "orc_tile2d_f32"):
                getattr(L, nm).argtypes = [fp, fp, fp, ctypes.c_int, ctypes.c_int, fp, fp, fp]
                getattr(L, nm).restype = None
            L.orc_tile_direct_f32.argtypes = [ctypes.c_int] * 3 + [fp, fp, fp]
            L.orc_tile_direct_f32.restype = None
            L.orc_wino_layer.argtypes = [fp, fp, fp] + [ctypes.c_int] * 7 + [dp] + [ctypes.c_int] * 3
            L.orc_wino_layer.restype = ctypes.c_int
            L.orc_wino_layer_tiles.argtypes = [fp, fp] + [ctypes.c_int] * 7 + [dp] + \
                [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int64), fp, ctypes.c_int]
            L.orc_wino_layer_tiles.restype = ctypes.c_int
            L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.orc_splitmix64.restype = ctypes.c_uint64
            L.orc_trial_value.argtypes = [ctypes.c_uint64] + [ctypes.c_int] * 5
            L.orc_trial_value.restype = ctypes.c_float
            L.orc_mask_points.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, ctypes.c_uint,
                                                              ctypes.c_double, dp]
            L.orc_mask_points.restype = ctypes.c_int
            L.orc_error_sweep.argtypes = [dp, ctypes.c_int, ctypes.POINTER(_Size), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_ubyte), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_uint64, dp, ctypes.c_int, ctypes.c_int]
            L.orc_error_sweep.restype = ctypes.c_int
            L.orc_direct_error.argtypes = [ctypes.c_int] * 4 + [ctypes.c_uint64]
            L.orc_direct_error.restype = ctypes.c_double
            L.orc_pointset_error.argtypes = [ctypes.c_int] * 3 + [dp, ctypes.c_int, ctypes.c_int,
                                                                  ctypes.c_uint64, dp]
            L.orc_pointset_error.restype = ctypes.c_int
            L.orc_tile2d_kron.argtypes = [dp, ctypes.c_int, ctypes.c_int, fp, fp, fp, ctypes.c_int]
            L.orc_tile2d_kron.restype = ctypes.c_int
            L.orc_pointset_error_kron.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_uint64, ctypes.c_int, dp]
            L.orc_pointset_error_kron.restype = ctypes.c_int
            ip = ctypes.POINTER(ctypes.c_int)
            L.orc_huffman_merges.argtypes = [dp, ctypes.c_int, ip, ip]
            L.orc_huffman_merges.restype = ctypes.c_int
            L.orc_huffman_dot_f32.argtypes = [fp, fp, ctypes.c_int]
            L.orc_huffman_dot_f32.restype = ctypes.c_float
            L.orc_tile_order.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, fp, fp, fp,
                                         ctypes.c_int]
            L.orc_tile_order.restype = ctypes.c_int
            L.orc_pointset_error_order.argtypes = [ctypes.c_int] * 3 + [
                dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, dp]
            L.orc_pointset_error_order.restype = ctypes.c_int
            L.orc_round_bf16.argtypes = [ctypes.c_float]
            L.orc_round_bf16.restype = ctypes.c_float
            L.orc_round_fp16.argtypes = [ctypes.c_float]
            L.orc_round_fp16.restype = ctypes.c_float
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class SingularPoints(ValueError):
    pass


def make_matrices(points, m: int, r: int):
    """FP64 (AT[m][alpha], G[alpha][r], BT[alpha][alpha]) in canonical order."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    a = m + r - 1
    if pts.size != a:
        raise ValueError("need alpha = m + r - 1 points")
    AT = np.zeros((m, a)); G = np.zeros((a, r)); BT = np.zeros((a, a))
    st = lib().orc_make_matrices(_dp(pts), m, r, _dp(AT), _dp(G), _dp(BT))
    if st == -2:
        raise SingularPoints("coinciding finite points")
    if st < 0:
        raise ValueError("invalid point set")
    return AT, G, BT


def canonical_points(points):
    pts = np.ascontiguousarray(points, dtype=np.float64)
    out = np.zeros_like(pts)
    if lib().orc_canonical_points(_dp(pts), pts.size, _dp(out)) < 0:
        raise ValueError("invalid point set")
    return out


def direct_f64(x, w, dim: int, pad: int, r: int):
    """FP64 direct correlation; x [N][C][(H)][W] and w [K][C][(r)][r] FP32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    if dim == 1:
        N, C, W = x.shape
        H = 1
        K = w.shape[0]
        y = np.zeros((N, K, W + 2 * pad - r + 1))
    else:
        N, C, H, W = x.shape
        K = w.shape[0]
        y = np.zeros((N, K, H + 2 * pad - r + 1, W + 2 * pad - r + 1))
    lib().orc_direct_f64(_fp(x), _fp(w), _dp(y), dim, N, C, K, H, W, pad, r)
    return y


def tile_f32(dim: int, AT, G, BT, m: int, r: int, g, d):
    AT = np.ascontiguousarray(AT, dtype=np.float32)
    G = np.ascontiguousarray(G, dtype=np.float32)
    BT = np.ascontiguousarray(BT, dtype=np.float32)
    g = np.ascontiguousarray(g, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float32)
    y = np.zeros(m if dim == 1 else m * m, dtype=np.float32)
    fn = lib().orc_tile1d_f32 if dim == 1 else lib().orc_tile2d_f32
    fn(_fp(AT), _fp(G), _fp(BT), m, r, _fp(g), _fp(d), _fp(y))
    return y if dim == 1 else y.reshape(m, m)


def tile_direct_f32(dim: int, m: int, r: int, g, d):
    g = np.ascontiguousarray(g, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float32)
    y = np.zeros(m if dim == 1 else m * m, dtype=np.float32)
    lib().orc_tile_direct_f32(dim, m, r, _fp(g), _fp(d), _fp(y))
    return y if dim == 1 else y.reshape(m, m)


LOWP = {"f32": 0, "bf16": 1, "fp16": 2, "split_bf16x3": 3, "split_bf16x6": 4}


def wino_layer(x, w, dim: int, pad: int, points, m: int, r: int, lowp: str = "f32"):
    """FP32 Winograd layer (oracle operation order); returns FP32 y."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if dim == 1:
        N, C, W = x.shape
        H = 1
        K = w.shape[0]
        y = np.zeros((N, K, W + 2 * pad - r + 1), dtype=np.float32)
    else:
        N, C, H, W = x.shape
        K = w.shape[0]
        y = np.zeros((N, K, H + 2 * pad - r + 1, W + 2 * pad - r + 1), dtype=np.float32)
    st = lib().orc_wino_layer(_fp(x), _fp(w), _fp(y), dim, N, C, K, H, W, pad, _dp(pts), m, r,
                              LOWP[lowp])
    if st == -2:
        raise SingularPoints("coinciding finite points")
    if st < 0:
        raise ValueError("invalid layer arguments")
    return y


def wino_layer_tiles(x, w, dim: int, pad: int, points, m: int, r: int, sel, lowp: str = "f32"):
    """Outputs of selected (tile, k) pairs of the layer (wino_layer's
    `lowp` modes): array [n_sel][m] (1D) or [n_sel][m][m] (2D), uncropped."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    pts = np.ascontiguousarray(points, dtype=np.float64)
    sel = np.ascontiguousarray(sel, dtype=np.int64).reshape(-1, 2)
    if dim == 1:
        N, C, W = x.shape
        H = 1
    else:
        N, C, H, W = x.shape
    K = w.shape[0]
    out = np.zeros((sel.shape[0],) + ((m,) if dim == 1 else (m, m)), dtype=np.float32)
    st = lib().orc_wino_layer_tiles(_fp(x), _fp(w), dim, N, C, K, H, W, pad, _dp(pts), m, r,
                                    sel.shape[0],
                                    sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _fp(out),
                                    LOWP[lowp])
    if st == -2:
        raise SingularPoints("coinciding finite points")
    if st < 0:
        raise ValueError("invalid arguments")
    return out


def splitmix64(seed: int, n: int) -> int:
    return int(lib().orc_splitmix64(seed & (2**64 - 1), n & (2**64 - 1)))


def trial_value(seed: int, dim: int, m: int, r: int, trial: int, idx: int) -> float:
    return float(lib().orc_trial_value(seed, dim, m, r, trial, idx))


def mask_points(dim: int, m: int, r: int, d: float, mask: int, c: float):
    out = np.zeros(16)
    n = lib().orc_mask_points(dim, m, r, d, mask, c, _dp(out))
    if n < 0:
        return None
    return out[:n].copy()


def error_sweep(c_grid, sizes, masks, trials: int, seed: int, c_stride: int = 1,
                n_threads: int = 1):
    """err[n_sizes][n_masks][n_c]; sizes = [(dim, m, r, d)].  Entries skipped by
    c_stride stay NaN."""
    cg = np.ascontiguousarray(c_grid, dtype=np.float64)
    sz = (_Size * len(sizes))(*[_Size(int(a), int(b), int(c), float(d)) for a, b, c, d in sizes])
    mk = np.ascontiguousarray(masks, dtype=np.uint8)
    err = np.full((len(sizes), mk.size, cg.size), np.nan)
    lib().orc_error_sweep(_dp(cg), cg.size, sz, len(sizes),
                          mk.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), mk.size, trials,
                          seed, _dp(err), c_stride, n_threads)
    return err


def tile2d_kron(points, m: int, r: int, g, d, pairwise: bool = False):
    """One 2D tile in the Kronecker-product form (Sec. 7): y [m][m]."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float32).ravel()
    d = np.ascontiguousarray(d, dtype=np.float32).ravel()
    y = np.zeros(m * m, np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    rc = lib().orc_tile2d_kron(_dp(pts), m, r, g.ctypes.data_as(fp), d.ctypes.data_as(fp),
                               y.ctypes.data_as(fp), int(pairwise))
    assert rc == 0, rc
    return y.reshape(m, m)


def pointset_error_kron(m: int, r: int, point_sets, trials: int, seed: int,
                        pairwise: bool = False):
    """The sweep metric of the Kronecker-product 2D form for explicit sets."""
    pts = np.ascontiguousarray(point_sets, dtype=np.float64)
    assert pts.ndim == 2 and pts.shape[1] == m + r - 1
    err = np.full(pts.shape[0], np.nan)
    rc = lib().orc_pointset_error_kron(m, r, _dp(pts), pts.shape[0], trials, seed, int(pairwise),
                                       _dp(err))
    assert rc == 0
    return err


ORDERS = {"fma": 0, "huffman": 1, "huffman_mixed": 2}


def huffman_merges(w):
    """Huffman tree over the leaves with w[k] > 0: list of (first, second)
    node ids per merge (leaf k = id k, merge s creates id len(w) + s)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros(len(w), np.int32)
    s = np.zeros(len(w), np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    n = lib().orc_huffman_merges(_dp(w), len(w), f.ctypes.data_as(ip), s.ctypes.data_as(ip))
    assert n >= 0
    return [(int(f[i]), int(s[i])) for i in range(n)]


def huffman_dot_f32(c, x) -> np.float32:
    """sum c[k] x[k] in FP32 along the Huffman tree of |c|."""
    c = np.ascontiguousarray(c, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    assert c.shape == x.shape and c.ndim == 1
    return np.float32(lib().orc_huffman_dot_f32(_fp(c), _fp(x), len(c)))


def tile_order(dim: int, points, m: int, r: int, g, d, order: str):
    """One tile in a summation-order variant ('huffman', 'huffman_mixed')."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float32).ravel()
    d = np.ascontiguousarray(d, dtype=np.float32).ravel()
    y = np.zeros(m if dim == 1 else m * m, np.float32)
    rc = lib().orc_tile_order(dim, _dp(pts), m, r, _fp(g), _fp(d), _fp(y), ORDERS[order])
    assert rc == 0, rc
    return y if dim == 1 else y.reshape(m, m)


def pointset_error_order(dim: int, m: int, r: int, point_sets, trials: int, seed: int,
                         order: str):
    """The sweep metric for explicit sets in one of the summation orders."""
    pts = np.ascontiguousarray(point_sets, dtype=np.float64)
    assert pts.ndim == 2 and pts.shape[1] == m + r - 1
    err = np.full(pts.shape[0], np.nan)
    rc = lib().orc_pointset_error_order(dim, m, r, _dp(pts), pts.shape[0], trials, seed,
                                        ORDERS[order], _dp(err))
    assert rc == 0
    return err


def direct_error(dim: int, m: int, r: int, trials: int, seed: int) -> float:
    return float(lib().orc_direct_error(dim, m, r, trials, seed))


def pointset_error(dim: int, m: int, r: int, point_sets, trials: int, seed: int):
    """The sweep metric of explicit point sets (each m + r - 1 values with one
    +inf, any order) on the sweep's trials of size (dim, m, r)."""
    pts = np.ascontiguousarray(point_sets, dtype=np.float64)
    assert pts.ndim == 2 and pts.shape[1] == m + r - 1
    err = np.full(pts.shape[0], np.nan)
    rc = lib().orc_pointset_error(dim, m, r, _dp(pts), pts.shape[0], trials, seed, _dp(err))
    assert rc == 0
    return err


def round_bf16(v: float) -> float:
    return float(lib().orc_round_bf16(v))


def round_fp16(v: float) -> float:
    return float(lib().orc_round_fp16(v))
