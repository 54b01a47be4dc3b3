"""wino_conv2d_f32_noalloc: the FP32 layer for callers that cannot allocate
device memory (code running under CUDA graph capture, plug-ins whose host
framework owns the memory pool).  It runs the same fused kernel as
wino_conv2d with its scratch in a fixed array inside the library, so its
output must equal the oracle's FP32 Winograd layer bit for bit -- the bar the
other FP32 layer tests use -- and wino_conv2d's, on consecutive calls that
reuse that array with different shapes.  Collected last (file name) so a
failure here leaves every other test already run."""
import ctypes
import math

import numpy as np
import pytest

from paper_2201_10369_gb300 import inputs

pytestmark = pytest.mark.gpu


def _noalloc(wino, x, w, y, pts, m, pad):
    """Calls the entry point through the C ABI directly."""
    import torch
    L = wino.load()
    N, C, H, W = x.shape
    K = w.shape[0]
    p = np.ascontiguousarray(pts, dtype=np.float64)
    st = L.wino_conv2d_f32_noalloc(x.data_ptr(), w.data_ptr(), y.data_ptr(), N, C, K, H, W, pad,
                                   p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), m, 3,
                                   torch.cuda.current_stream().cuda_stream)
    return st


def test_noalloc_matches_oracle_and_conv2d_on_consecutive_calls(wino, orc):
    import torch
    c = 1.622
    cases = [((2, 24, 64, 30, 21, 1), 4, [0.0, -1 / c, -c, c, 1 / c, math.inf]),
             ((1, 40, 128, 17, 17, 1), 6, [0.0, -0.5, -2.0, 2.0, 0.5, -1.003, 1.003, math.inf]),
             ((3, 8, 64, 12, 9, 0), 2, [0.0, 1.0, -1.0, math.inf])]
    for (N, C, K, H, W, pad), m, pts in cases:
        x, w = inputs.layer_uniform(N, C, K, H, W, seed=N + C + K)
        xt, wt = torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda()
        shape = (N, K, H + 2 * pad - 2, W + 2 * pad - 2)
        yo = orc.wino_layer(x, w, 2, pad, pts, m, 3)
        ref = torch.full(shape, float("nan"), device="cuda")
        wino.wino_conv2d(xt, wt, ref, pts, m, 3, pad)
        for _ in range(2):
            y = torch.full(shape, float("nan"), device="cuda")
            assert _noalloc(wino, xt, wt, y, pts, m, pad) == wino.WINO_OK, wino.wino_last_error()
            torch.cuda.synchronize()
            assert np.array_equal(y.cpu().numpy(), yo)
            assert torch.equal(y, ref)


def test_noalloc_rejects_oversized_and_unsupported(wino):
    import torch
    x = torch.zeros((1, 512, 8, 8), device="cuda")
    w = torch.zeros((512, 512, 3, 3), device="cuda")
    y = torch.zeros((1, 512, 8, 8), device="cuda")
    pts = [0.0, -0.5, -2.0, 2.0, 0.5, math.inf]
    assert _noalloc(wino, x, w, y, pts, 4, 1) == wino.WINO_EINVAL  # 36 * 512 * 512 > 4 Mi
    assert "scratch" in wino.wino_last_error()
    w2 = torch.zeros((48, 512, 3, 3), device="cuda")
    y2 = torch.zeros((1, 48, 8, 8), device="cuda")
    assert _noalloc(wino, x, w2, y2, pts, 4, 1) == wino.WINO_EINVAL  # K not a multiple of 64
