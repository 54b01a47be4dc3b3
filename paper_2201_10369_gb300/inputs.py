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


# The comparison point sets of Barabasz et al. that Tables 7 (1D) and 8 (2D)
# list beside the proposed ones, finite points of F(n - 2, 3) (infinity is
# the extra point), keyed (dim, n); and the paper's improvement (%) of its
# proposed set over each (Tables 7-8, last column).
_P4 = [0.0, -1.0, 1.0]
COMPARISON_SETS = {
    (1, 4): _P4, (1, 5): _P4 + [0.5], (1, 6): _P4 + [0.5, -3.0],
    (1, 7): _P4 + [0.5, -0.5, -3.0], (1, 8): _P4 + [0.5, -0.5, 2.0, -2.0],
    (1, 9): _P4 + [0.5, -0.5, 2.0, -2.0, -0.25], (1, 10): _P4 + [0.5, -0.5, 2.0, -2.0, -0.25, 4.0],
    (2, 4): _P4, (2, 5): _P4 + [0.5], (2, 6): _P4 + [0.5, -2.0],
    (2, 7): _P4 + [0.5, -2.0, -0.5], (2, 8): _P4 + [0.5, -0.5, 2.0, -2.0],
    (2, 9): _P4 + [0.5, -0.5, 2.0, -2.0, -0.25], (2, 10): _P4 + [0.5, -0.5, 2.0, -2.0, -0.25, 4.0],
}
def _cd(c, d, slots):
    """Points named by slot letters: z 0, a -1/c, b -c, C c, A 1/c, e -1/d,
    f -d, D d, E 1/d, p +1, m -1, h 1/2."""
    v = {"z": 0.0, "a": -1.0 / c, "b": -c, "C": c, "A": 1.0 / c, "p": 1.0, "m": -1.0,
         "h": 0.5}
    if d is not None:
        v.update({"e": -1.0 / d, "f": -d, "D": d, "E": 1.0 / d})
    return [v[k] for k in slots]


# The paper's proposed point sets (Tables 7-8, "Proposed points" column),
# finite points keyed (dim, n).
PROPOSED_SETS = {
    (1, 4): _cd(1.028, None, "zmA"), (1, 5): _cd(1.5, None, "zhbC"),
    (1, 6): _cd(1.829, None, "abzCA"), (1, 7): _cd(2.22, 1.0, "zabCAD"),
    (1, 8): _cd(2.0, 1.0, "zabCAfD"), (1, 9): _cd(1.313, 2.478, "zabCAefD"),
    (1, 10): _cd(1.953, 1.229, "abefzCDEA"),
    (2, 4): _cd(1.054, None, "zaA"), (2, 5): _cd(2.0, None, "zpmb"),
    (2, 6): _cd(1.622, None, "abzCA"), (2, 7): _cd(2.0, 1.0, "zabCAD"),
    (2, 8): _cd(2.0, 1.003, "zabCAeD"), (2, 9): _cd(1.305, 2.485, "zabCAefD"),
    (2, 10): _cd(1.272, 2.099, "abefzCDEA"),
}
PAPER_IMPROVEMENT_PCT = {
    (1, 4): -24.9, (1, 5): 9.6, (1, 6): 18.35, (1, 7): -14.44, (1, 8): 0.0, (1, 9): 2.14,
    (1, 10): 59.54, (2, 4): -20.52, (2, 5): 35.75, (2, 6): 27.96, (2, 7): -13.36, (2, 8): 0.0,
    (2, 9): 17.5, (2, 10): 28.16,
}


def chebyshev_points(n):
    """The n Chebyshev nodes cos((2k - 1) pi / (2 n)), k = 1..n (Sec. 2), as
    finite points (infinity is added as the extra point)."""
    k = np.arange(1, n + 1)
    return list(np.cos((2 * k - 1) / (2 * n) * np.pi))
