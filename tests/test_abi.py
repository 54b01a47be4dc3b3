"""CPU checks of the C ABI: the library builds and loads, exports every
symbol include/wino.h declares, and its host-only logic (FP64 matrix
construction, argument validation) behaves.  No device compute here."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2201_10369_gb300 as w
    w.build()
    return w


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(wino_[a-z0-9_]+)\s*\(", src, re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "wino_conv2d" in names and "wino_error_sweep" in names and len(names) >= 12
    L = lib.load()
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("m,r", [(2, 3), (4, 3), (6, 3), (8, 3), (2, 5), (6, 5)])
def test_host_matrices_match_oracle(lib, orc, m, r):
    """Host FP64 construction vs the oracle's: same definition, same rounding
    order, so bit-identical (the parity bar is 1e-13 relative)."""
    rng = np.random.default_rng(m * 10 + r)
    pts = list(rng.uniform(-3, 3, m + r - 2)) + [math.inf]
    got = lib.wino_make_matrices(pts, m, r)
    want = orc.make_matrices(pts, m, r)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def test_host_validation(lib):
    with pytest.raises(lib.WinoError) as e:
        lib.wino_make_matrices([0.0, 1.0, 1.0, math.inf], 2, 3)
    assert e.value.status == lib.WINO_ESINGULAR
    for bad in ([0.0, 1.0, -1.0, 2.0], [0.0, math.nan, 1.0, math.inf], [0.0, -math.inf, 1, 2]):
        with pytest.raises(lib.WinoError) as e:
            lib.wino_make_matrices(bad, 2, 3)
        assert e.value.status == lib.WINO_EINVAL
    assert lib.wino_workspace_bytes(1, 8, 8, 16, 16, 2, 3) > 0
    assert lib.wino_workspace_bytes(1, 8, 8, 2, 2, 2, 9) == 0


def test_no_cpu_fallback(lib):
    """Without a GPU every device entry point refuses (WINO_EUNSUPPORTED)
    instead of computing anything on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert not lib.wino_device_ok()
    L = lib.load()
    pts = np.array([0.0, 1.0, -1.0, math.inf])
    st = L.wino_conv2d(16, 16, 16, 1, 2, 2, 8, 8, 1, pts.ctypes.data_as(lib._DP), 2, 3, 0, None)
    assert st == lib.WINO_EUNSUPPORTED
    with pytest.raises(lib.WinoError) as e:
        lib.wino_error_sweep([1.5], [(1, 2, 3, 1.0)], [0x06], 10, 0, stream=0)
    assert e.value.status == lib.WINO_EUNSUPPORTED


def test_pointset_validation_on_host(wino):
    """A point set without exactly one +inf is rejected before any device
    work (and without writing past the caller's set)."""
    import ctypes
    import math
    L = wino.load()
    pts = (ctypes.c_double * 8)(0.0, 1.0, -1.0, 2.0, 0.0, 1.0, -1.0, math.inf)
    err = (ctypes.c_double * 2)()
    assert L.wino_pointset_error(1, 2, 3, pts, 2, 10, 0, err, None) == wino.WINO_EINVAL
    pts2 = (ctypes.c_double * 4)(0.0, math.inf, -1.0, math.inf)
    assert L.wino_pointset_error(1, 2, 3, pts2, 1, 10, 0, err, None) == wino.WINO_EINVAL


def test_order_validation_on_host(wino):
    """An order outside WINO_ORDER_FMA .. WINO_ORDER_HUFFMAN_MIXED is rejected
    before any device work, by both order entry points."""
    import ctypes
    import math
    L = wino.load()
    pts = (ctypes.c_double * 4)(0.0, 1.0, -1.0, math.inf)
    err = (ctypes.c_double * 1)()
    for order in (-1, 3):
        assert L.wino_pointset_error_order(1, 2, 3, pts, 1, 10, 0, order, err,
                                           None) == wino.WINO_EINVAL
        cg = (ctypes.c_double * 1)(2.0)
        sz = (wino.WinoSize * 1)(wino.WinoSize(1, 2, 3, 1.0))
        mk = (ctypes.c_ubyte * 1)(0x60)
        assert L.wino_error_sweep_order(cg, 1, sz, 1, mk, 1, 10, 0, order, err,
                                        None) == wino.WINO_EINVAL
    assert "order" in wino.wino_last_error()


def test_wait_probe_validation_on_host(wino):
    """wino_wait_probe rejects a NULL result pointer or a poll count below 1
    before any device work; WINO_WAIT_POLLS is the layer kernels' limit."""
    import ctypes
    import pathlib
    import re
    L = wino.load()
    ns = ctypes.c_longlong(0)
    assert L.wino_wait_probe(0, ctypes.byref(ns), None) == wino.WINO_EINVAL
    assert L.wino_wait_probe(16, None, None) == wino.WINO_EINVAL
    hdr = (pathlib.Path(__file__).resolve().parents[1] / "include" / "wino.h").read_text()
    m = re.search(r"#define WINO_WAIT_POLLS \(1 << (\d+)\)", hdr)
    assert m and 1 <= int(m.group(1)) <= 24


def test_binding_validates_arguments_before_the_abi(lib):
    """The Python wrappers check dtype, shapes and the point count before any
    ABI call (the library indexes device memory from the sizes alone), so a
    wrong argument raises ValueError and never reaches a kernel.  CPU
    tensors: every check up to the device one runs here."""
    import torch
    pts4 = [0.0, 1.0, -1.0, math.inf]
    x = torch.zeros((1, 8, 6, 6))
    w = torch.zeros((16, 8, 3, 3))
    y = torch.zeros((1, 16, 6, 6))
    cases = [
        (x.double(), w, y, pts4, "x must be torch.float32"),
        (x, w.to(torch.bfloat16), y, pts4, "w must be torch.float32"),
        (x, torch.zeros((16, 4, 3, 3)), y, pts4, "w must have shape"),
        (x, w, torch.zeros((1, 16, 5, 6)), pts4, "y must have shape"),
        (x, w, torch.zeros((1, 8, 6, 6)), pts4, "y must have shape"),
        (x, w, y, pts4[:3], "need alpha"),
        (x[0], w, y, pts4, "dimensions"),
    ]
    for xa, wa, ya, p, msg in cases:
        with pytest.raises(ValueError, match=msg):
            lib.wino_conv2d(xa, wa, ya, p, 2, 3, 1)
    with pytest.raises(ValueError, match="need alpha"):
        lib.wino_conv2d_f32_noalloc(x, w, y, pts4 + [2.0], 2, 3, 1)
    with pytest.raises(ValueError, match="y must have shape"):
        lib.wino_conv1d(torch.zeros((2, 8, 10)), torch.zeros((4, 8, 3)), torch.zeros((2, 4, 9)),
                        pts4, 2, 3, 1)
    with pytest.raises(ValueError, match="y64 must be torch.float64"):
        lib.wino_direct_conv_f64(x, w, y, 1)
    with pytest.raises(ValueError, match="same number"):
        lib.wino_error_stats(y, torch.zeros(5, dtype=torch.float64))
    # well-formed CPU tensors pass every check but the device one
    with pytest.raises(ValueError, match="CUDA tensor"):
        lib.wino_conv2d(x, w, y, pts4, 2, 3, 1)
