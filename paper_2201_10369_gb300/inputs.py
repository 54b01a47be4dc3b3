"""Seeded synthetic workloads shaped like the paper's (Sec. 6: uniform random
inputs; Sec. 6.4: CNN layers).  No arithmetic of the method lives here: this
module only draws inputs and names workload shapes, so the GPU path and the
CPU oracle can be fed the same arrays.

- layer inputs: x, w i.i.d. uniform [-1, 1) (numpy PCG64, `seed`);
- VGG16-shaped 3x3 layers: x = ReLU(N(0, 1)), w ~ N(0, 2 / (9 C)) (He normal);
- the sweep grid: c_k = 0.05 * 400^(k / 4095), k < 4096 (log-spaced over
  [0.05, 20]); 1D F(m,3) m = 2..8 and 2D F(m x m,3x3) m = 2..6 with the fixed
  d of the paper's Tables 7-8 for 1D F(7,3) / F(8,3); the subsets of the slots
  [-1/c, -c, c, 1/c, -1/d, -d, d, 1/d] the sweep visits.
"""
from __future__ import annotations

import numpy as np

# VGG16's 3x3 convolution shapes by stage (C_in = C_out, H = W); batch 32.
VGG16_LAYERS = [(64, 224), (128, 112), (256, 56), (512, 28), (512, 14)]
VGG_BATCH = 32

SWEEP_TRIALS = 1000
SWEEP_NC = 4096


def uniform_pm1(shape, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape).astype(np.float32)


def layer_uniform(N, C, K, H, W, r=3, seed: int = 0, dim: int = 2):
    """(x, w) uniform in [-1, 1); x drawn first, then w, from one stream."""
    rng = np.random.default_rng(seed)
    if dim == 1:
        x = rng.uniform(-1.0, 1.0, size=(N, C, W)).astype(np.float32)
        w = rng.uniform(-1.0, 1.0, size=(K, C, r)).astype(np.float32)
    else:
        x = rng.uniform(-1.0, 1.0, size=(N, C, H, W)).astype(np.float32)
        w = rng.uniform(-1.0, 1.0, size=(K, C, r, r)).astype(np.float32)
    return x, w


def vgg_layer_host(C, H, N=VGG_BATCH, seed: int = 0, r=3):
    """x = ReLU(N(0,1)) [N][C][H][H], w ~ N(0, 2/(9C)) [C][C][r][r] (FP32)."""
    rng = np.random.default_rng(seed)
    x = np.maximum(rng.standard_normal((N, C, H, H), dtype=np.float32), 0.0)
    w = (rng.standard_normal((C, C, r, r), dtype=np.float32) *
         np.float32(np.sqrt(2.0 / (r * r * C))))
    return x, w


def vgg_layer_device(C, H, N=VGG_BATCH, seed: int = 0, r=3, device="cuda"):
    """Same distribution drawn with torch's generator on the device (fast for
    the full batch); returns CUDA tensors."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.randn((N, C, H, H), generator=g, device=device, dtype=torch.float32).clamp_(min=0)
    w = torch.randn((C, C, r, r), generator=g, device=device, dtype=torch.float32)
    w.mul_(float(np.sqrt(2.0 / (r * r * C))))
    return x, w


def c_grid(n: int = SWEEP_NC, lo: float = 0.05, hi: float = 20.0) -> np.ndarray:
    k = np.arange(n, dtype=np.float64)
    return lo * (hi / lo) ** (k / (n - 1))


# (dim, m, r, d): the sweep's problem sizes.
SWEEP_SIZES = ([(1, m, 3, 1.0) for m in range(2, 7)] + [(1, 7, 3, 2.478), (1, 8, 3, 1.229)] +
               [(2, m, 3, 1.0) for m in range(2, 7)])


def sweep_masks() -> np.ndarray:
    """Subsets visited: 2..6 of the six slots {-1/c, -c, c, 1/c, -1, 1} (bits
    0-3, 5, 6), plus 7 or 8 of all eight slots (sizes with a free d)."""
    out = []
    for mk in range(1, 256):
        pc = bin(mk).count("1")
        if 2 <= pc <= 6 and not (mk & 0x90):
            out.append(mk)
        elif pc >= 7:
            out.append(mk)
    return np.array(out, dtype=np.uint8)
