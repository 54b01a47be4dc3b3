"""Pins of the oracle's direct correlation and FP32 Winograd (Eqs. (1), (8),
(9)) against exact rational arithmetic, brute force, exactly representable
cases and error bounds."""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import rational as R


def test_direct_f64_vs_rational_bruteforce(orc):
    """Inputs on a 2^-4 grid make every FP64 product and sum exact, so the
    FP64 direct correlation must equal the rational brute force exactly."""
    rng = np.random.default_rng(1)
    x = (rng.integers(-32, 32, size=(2, 2, 5, 5)) / 16.0).astype(np.float32)
    w = (rng.integers(-32, 32, size=(3, 2, 3, 3)) / 16.0).astype(np.float32)
    y = orc.direct_f64(x, w, 2, 1, 3)
    yq = R.direct_layer_2d(x.tolist(), w.tolist(), 1)
    assert np.array_equal(y, np.array([[[[float(v) for v in row] for row in ch] for ch in n]
                                       for n in yq]))


def test_direct_f64_delta_kernel(orc):
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, size=(1, 3, 7, 6)).astype(np.float32)
    w = np.zeros((3, 3, 3, 3), np.float32)
    for k in range(3):
        w[k, k, 1, 1] = 1.0
    assert np.array_equal(orc.direct_f64(x, w, 2, 1, 3), x.astype(np.float64))
    x1 = x[:, :, 0, :]
    w1 = np.zeros((3, 3, 3), np.float32)
    for k in range(3):
        w1[k, k, 1] = 1.0
    assert np.array_equal(orc.direct_f64(x1, w1, 1, 1, 3), x1.astype(np.float64))


@pytest.mark.parametrize("r", [3, 5])
@pytest.mark.parametrize("m", range(2, 9))
def test_winograd_exact_in_rationals(m, r):
    """Toom-Cook is exact (Sec. 4): rational Winograd equals rational
    correlation for 1D and 2D tiles."""
    alpha = m + r - 1
    if alpha > 10:
        pytest.skip("alpha > 10 not used")
    rng = random.Random(m * 31 + r)
    pts = set()
    while len(pts) < alpha - 1:
        pts.add(Fraction(rng.randint(-9, 9), rng.randint(1, 4)))
    AT, G, BT = R.matrices(sorted(pts) + ["inf"], m, r)
    g = [Fraction(rng.randint(-5, 5)) for _ in range(r)]
    d = [Fraction(rng.randint(-5, 5)) for _ in range(alpha)]
    assert R.wino_tile_1d(AT, G, BT, g, d) == R.correlate_1d(g, d)
    if alpha <= 8:
        g2 = [[Fraction(rng.randint(-3, 3)) for _ in range(r)] for _ in range(r)]
        d2 = [[Fraction(rng.randint(-3, 3)) for _ in range(alpha)] for _ in range(alpha)]
        assert R.wino_tile_2d(AT, G, BT, g2, d2) == R.correlate_2d(g2, d2)


def test_fp32_tile_exact_for_lavin_points(orc):
    """With points {0, 1, -1, inf} every FP32 intermediate of F(2,3) and
    F(2x2,3x3) on small integers is exact, so the FP32 tile must equal the
    exact correlation: a transposed operand or a wrong index fails here."""
    AT, G, BT = orc.make_matrices([0.0, 1.0, -1.0, math.inf], 2, 3)
    rng = np.random.default_rng(3)
    for _ in range(50):
        g = rng.integers(-8, 9, size=3).astype(np.float32)
        d = rng.integers(-8, 9, size=4).astype(np.float32)
        y = orc.tile_f32(1, AT, G, BT, 2, 3, g, d)
        assert np.array_equal(y, [sum(g[k] * d[j + k] for k in range(3)) for j in range(2)])
        g2 = rng.integers(-8, 9, size=(3, 3)).astype(np.float32)
        d2 = rng.integers(-8, 9, size=(4, 4)).astype(np.float32)
        y2 = orc.tile_f32(2, AT, G, BT, 2, 3, g2, d2)
        want = [[float((g2 * d2[a:a + 3, b:b + 3]).sum()) for b in range(2)] for a in range(2)]
        assert np.array_equal(y2, want)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("m", [2, 4, 6])
def test_fp32_tile_error_bound(orc, dim, m):
    """FP32 Winograd of one tile lies within a first-order error bound of the
    FP64 correlation: |yhat - y| <= gamma * (|AT| (|G||g| .* |BT||d|)) with
    gamma = (terms) * 2^-24, the standard bound for nested dot products."""
    c = 1.6
    base = [-1 / c, -c, c, 1 / c, -1.0, 1.0][:m]
    pts = [0.0] + base + [math.inf]
    ATd, Gd, BTd = orc.make_matrices(pts, m, 3)
    AT, G, BT = (a.astype(np.float32) for a in (ATd, Gd, BTd))
    rng = np.random.default_rng(4)
    a = m + 2
    u = 2.0 ** -24
    for _ in range(20):
        if dim == 1:
            g = rng.uniform(-1, 1, 3).astype(np.float32)
            d = rng.uniform(-1, 1, a).astype(np.float32)
            y = orc.tile_f32(1, AT, G, BT, m, 3, g, d).astype(np.float64)
            ref = np.array([np.dot(g.astype(np.float64), d[j:j + 3]) for j in range(m)])
            bound = np.abs(AT) @ ((np.abs(G) @ np.abs(g)) * (np.abs(BT) @ np.abs(d)))
            gamma = (3 + a + a + 2) * u
        else:
            g = rng.uniform(-1, 1, (3, 3)).astype(np.float32)
            d = rng.uniform(-1, 1, (a, a)).astype(np.float32)
            y = orc.tile_f32(2, AT, G, BT, m, 3, g, d).astype(np.float64)
            ref = np.array([[(g.astype(np.float64) * d[i:i + 3, j:j + 3]).sum() for j in range(m)]
                            for i in range(m)])
            aG, aB, aA = np.abs(G), np.abs(BT), np.abs(AT)
            bound = aA @ ((aG @ np.abs(g) @ aG.T) * (aB @ np.abs(d) @ aB.T)) @ aA.T
            gamma = 2 * (3 + a + a + 2) * u
        assert np.all(np.abs(y - ref) <= gamma * bound + 1e-30)


def test_layer_exact_case_and_ragged_tiles(orc):
    """Integer inputs with points {0, 1, -1, inf}: the FP32 layer is exact, so
    it must reproduce the FP64 direct correlation bit for bit, including the
    zero padding and the ragged last tile row/column (Ho = Wo = 15, m = 2)."""
    rng = np.random.default_rng(5)
    x = rng.integers(-4, 5, size=(2, 3, 15, 15)).astype(np.float32)
    w = rng.integers(-2, 3, size=(4, 3, 3, 3)).astype(np.float32)
    y = orc.wino_layer(x, w, 2, 1, [0.0, 1.0, -1.0, math.inf], 2, 3)
    assert np.array_equal(y.astype(np.float64), orc.direct_f64(x, w, 2, 1, 3))
    x1 = rng.integers(-4, 5, size=(2, 3, 23)).astype(np.float32)
    w1 = rng.integers(-2, 3, size=(4, 3, 3)).astype(np.float32)
    y1 = orc.wino_layer(x1, w1, 1, 1, [0.0, 1.0, -1.0, math.inf], 2, 3)
    assert np.array_equal(y1.astype(np.float64), orc.direct_f64(x1, w1, 1, 1, 3))


def test_layer_single_channel_equals_tile(orc):
    """C = K = 1, one tile: the layer oracle and the tile oracle agree bit for
    bit (the contraction over one channel is the Hadamard product)."""
    rng = np.random.default_rng(6)
    c = 1.829
    pts = [0.0, -1 / c, -c, c, 1 / c, math.inf]
    ATd, Gd, BTd = orc.make_matrices(pts, 4, 3)
    AT, G, BT = (a.astype(np.float32) for a in (ATd, Gd, BTd))
    d = rng.uniform(-1, 1, (6, 6)).astype(np.float32)
    g = rng.uniform(-1, 1, (3, 3)).astype(np.float32)
    y = orc.wino_layer(d.reshape(1, 1, 6, 6), g.reshape(1, 1, 3, 3), 2, 0, pts, 4, 3)
    assert np.array_equal(y.reshape(4, 4), orc.tile_f32(2, AT, G, BT, 4, 3, g, d))


@pytest.mark.parametrize("m,c", [(2, None), (4, 1.622), (6, 2.0)])
def test_layer_error_scale(orc, m, c):
    """The FP32 layer's relative L1 error vs FP64 direct is at the FP32
    Winograd scale (well below 1e-5) and above the direct-FP32 floor."""
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, (1, 8, 16, 16)).astype(np.float32)
    w = rng.uniform(-1, 1, (8, 8, 3, 3)).astype(np.float32)
    if c is None:
        pts = [0.0, -1.0, 1.0, math.inf]
    else:
        pts = [0.0, -1 / c, -c, c, 1 / c, -1.0, 1.0][: m + 1] + [math.inf]
    y = orc.wino_layer(x, w, 2, 1, pts, m, 3).astype(np.float64)
    ref = orc.direct_f64(x, w, 2, 1, 3)
    e = np.abs(y - ref).sum() / np.abs(ref).sum()
    assert 1e-9 < e < 1e-5


def test_round_bf16_fp16_vs_library(orc):
    """Operand rounding of the precision form against library conversions
    (numpy float16 and torch bfloat16 both round to nearest even)."""
    import torch
    rng = np.random.default_rng(8)
    vals = np.concatenate([rng.normal(0, 1, 2000), rng.normal(0, 1e-5, 500),
                           rng.normal(0, 3e4, 500), [65519.0, 65520.0, 6e-8, 1 + 2 ** -8,
                                                     1 + 3 * 2 ** -9]]).astype(np.float32)
    for v in vals:
        with np.errstate(over="ignore"):  # 65520 and above round to FP16 infinity
            want16 = float(np.float16(v))
        assert orc.round_fp16(float(v)) == want16
        assert orc.round_bf16(float(v)) == float(torch.tensor(float(v)).to(torch.bfloat16).float())


def test_lowp_layer_error_ordering(orc):
    """Reduced-precision contraction: BF16 error is far above FP32's, FP16 is
    below BF16, and split BF16x3 recovers most of the gap (Sec. 6 metric)."""
    rng = np.random.default_rng(9)
    x = np.maximum(rng.normal(0, 1, (1, 16, 12, 12)), 0).astype(np.float32)
    w = rng.normal(0, math.sqrt(2 / (9 * 16)), (16, 16, 3, 3)).astype(np.float32)
    c = 1.622
    pts = [0.0, -1 / c, -c, c, 1 / c, math.inf]
    ref = orc.direct_f64(x, w, 2, 1, 3)
    err = {}
    for mode in ("f32", "bf16", "fp16", "split_bf16x3"):
        y = orc.wino_layer(x, w, 2, 1, pts, 4, 3, mode).astype(np.float64)
        err[mode] = np.abs(y - ref).sum() / np.abs(ref).sum()
    assert err["f32"] < 1e-6
    assert err["bf16"] > 20 * err["f32"]
    assert err["fp16"] < err["bf16"]
    assert err["split_bf16x3"] < err["bf16"] / 20


@pytest.mark.parametrize("xs,ws,C", [(1000, 300, 1), (200, 200, 3)])
def test_split_bf16x6_exact_on_integer_operands(orc, xs, ws, C):
    """Exact regime: integer inputs and the points {0, -1, 1, inf} (exact FP32
    matrices) keep every FP32 step of the layer exact, so the FP32 layer
    equals the FP64 direct correlation.  The three-part split holds every bit
    of each operand and keeps every nonzero product of operands with at most
    16 significant bits, so split BF16x6 must reproduce it bit for bit, while
    split BF16x3 (lo x lo dropped) must not -- a dropped or misplaced part or
    product fails here."""
    rng = np.random.default_rng(5)
    x = rng.integers(-xs, xs + 1, (1, C, 8, 8)).astype(np.float32)
    w = rng.integers(-ws, ws + 1, (2, C, 3, 3)).astype(np.float32)
    pts = [0.0, -1.0, 1.0, math.inf]
    ref = orc.direct_f64(x, w, 2, 1, 3)
    y32 = orc.wino_layer(x, w, 2, 1, pts, 2, 3, "f32")
    assert np.array_equal(y32.astype(np.float64), ref)
    assert np.array_equal(orc.wino_layer(x, w, 2, 1, pts, 2, 3, "split_bf16x6"), y32)
    assert not np.array_equal(orc.wino_layer(x, w, 2, 1, pts, 2, 3, "split_bf16x3"), y32)


@pytest.mark.parametrize("C,H,m", [(16, 12, 4), (64, 20, 6)])
def test_split_bf16x6_error_not_above_fp32(orc, C, H, m):
    """Split BF16x6 with its two accumulators (hh alone; the five small
    products apart) is at least as accurate against FP64 as the FP32 layer."""
    from paper_2201_10369_gb300 import inputs
    x, w = inputs.vgg_layer_host(C, H, N=2, seed=3)
    c = 1.622
    pts = {4: [0.0, -1 / c, -c, c, 1 / c, math.inf],
           6: [0.0, -0.5, -2.0, 2.0, 0.5, -1.003, 1.003, math.inf]}[m]
    ref = orc.direct_f64(x, w, 2, 1, 3)
    err = {}
    for mode in ("f32", "split_bf16x6"):
        y = orc.wino_layer(x, w, 2, 1, pts, m, 3, mode).astype(np.float64)
        err[mode] = np.abs(y - ref).sum() / np.abs(ref).sum()
    assert err["split_bf16x6"] <= err["f32"], err


@pytest.mark.parametrize("dim,m", [(2, 2), (2, 4), (2, 6), (1, 4)])
@pytest.mark.parametrize("lowp", ["f32", "bf16", "fp16", "split_bf16x3", "split_bf16x6"])
def test_layer_tiles_equals_layer(orc, dim, m, lowp):
    """The per-tile oracle entry reproduces the full layer bit for bit on
    every (tile, k) of a small ragged layer, in every precision mode (the
    per-tile scales are the whole layer's)."""
    rng = np.random.default_rng(20 + m)
    c = 1.7
    pts = [0.0, -1 / c, -c, c, 1 / c, -1.0, 1.0][: m + 1] + [math.inf]
    if dim == 2:
        x = rng.uniform(-1, 1, (2, 3, 11, 9)).astype(np.float32)
        w = rng.uniform(-1, 1, (4, 3, 3, 3)).astype(np.float32)
    else:
        x = rng.uniform(-1, 1, (2, 3, 19)).astype(np.float32)
        w = rng.uniform(-1, 1, (4, 3, 3)).astype(np.float32)
    y = orc.wino_layer(x, w, dim, 1, pts, m, 3, lowp)
    Ho = 1 if dim == 1 else y.shape[2]
    Wo = y.shape[-1]
    th, tw = (1 if dim == 1 else -(-Ho // m)), -(-Wo // m)
    sel = [(t, k) for t in range(2 * th * tw) for k in range(4)]
    out = orc.wino_layer_tiles(x, w, dim, 1, pts, m, 3, sel, lowp)
    for (t, k), o in zip(sel, out):
        n, ti, tj = t // (th * tw), (t // tw) % th, t % tw
        if dim == 1:
            for b in range(m):
                if tj * m + b < Wo:
                    assert o[b] == y[n, k, tj * m + b]
        else:
            for a in range(m):
                for b in range(m):
                    if ti * m + a < Ho and tj * m + b < Wo:
                        assert o[a, b] == y[n, k, ti * m + a, tj * m + b]
