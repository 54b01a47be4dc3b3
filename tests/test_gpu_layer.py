"""GPU parity of the Winograd layer (wino_conv2d / wino_conv1d, FP32 form)
and of the FP64 reference / error-reduction kernels, through the C ABI,
element by element against the CPU oracle on the same seeded inputs."""
import math

import numpy as np
import pytest

from paper_2201_10369_gb300 import inputs

pytestmark = pytest.mark.gpu

LAVIN = [0.0, 1.0, -1.0, math.inf]


def full_group(c, extra=()):
    return [0.0, -1 / c, -c, c, 1 / c, *extra, math.inf]


POINTS = {
    2: LAVIN,
    4: full_group(1.622),
    6: full_group(2.0, (-1.0, 1.0)),  # P8 = {0, +-1/2, +-1, +-2, inf}
}


def _run2d(wino, x, w, pts, m, pad, dtype="f32"):
    import torch
    xt = torch.from_numpy(x).cuda()
    wt = torch.from_numpy(w).cuda()
    N, C, H, W = x.shape
    K, r = w.shape[0], w.shape[-1]
    y = torch.full((N, K, H + 2 * pad - r + 1, W + 2 * pad - r + 1), float("nan"),
                   device="cuda")
    wino.wino_conv2d(xt, wt, y, pts, m, r, pad, dtype)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_config1_f2x2_layer(wino, orc):
    """F(2x2,3x3), points {0,1,-1,inf}, N=1, C=K=8, 16x16, pad 1, uniform
    inputs from seed 0: bit-identical to the oracle, and at the FP32 error
    scale against FP64 direct correlation."""
    x, w = inputs.layer_uniform(1, 8, 8, 16, 16, seed=0)
    y = _run2d(wino, x, w, LAVIN, 2, 1)
    yo = orc.wino_layer(x, w, 2, 1, LAVIN, 2, 3)
    assert np.array_equal(y, yo)
    ref = orc.direct_f64(x, w, 2, 1, 3)
    rel = np.abs(y - ref).sum() / np.abs(ref).sum()
    assert rel < 1e-6
    assert np.abs(y - ref).max() / np.abs(ref).max() < 2e-6


@pytest.mark.parametrize("m", [2, 4, 6])
@pytest.mark.parametrize("shape", [(2, 5, 3, 15, 17, 1), (1, 16, 70, 9, 8, 2), (1, 1, 1, 3, 3, 0),
                                   (3, 9, 12, 13, 6, 1)])
def test_layer_bitwise_vs_oracle(wino, orc, m, shape):
    """Ragged tiles, channel counts off the kernels' blocking, padding 0-2."""
    N, C, K, H, W, pad = shape
    x, w = inputs.layer_uniform(N, C, K, H, W, seed=m)
    y = _run2d(wino, x, w, POINTS[m], m, pad)
    yo = orc.wino_layer(x, w, 2, pad, POINTS[m], m, 3)
    assert np.array_equal(y, yo)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6])
def test_layer_5x5_bitwise_vs_oracle(wino, orc, m):
    """The 5x5-kernel column of Table 1: F(m x m, 5 x 5), alpha = m + 4 up to 10,
    pad 2, ragged tiles: bit-identical to the oracle and at the FP32 error scale
    against FP64 direct correlation."""
    x, w = inputs.layer_uniform(2, 6, 5, 19, 14, r=5, seed=20 + m)
    pts = [0.0, -0.5, 0.5, -2.0, 2.0, -1.0, 1.0, -0.25, 4.0][: m + 3] + [math.inf]
    y = _run2d(wino, x, w, pts, m, 2)
    assert np.array_equal(y, orc.wino_layer(x, w, 2, 2, pts, m, 5))
    ref = orc.direct_f64(x, w, 2, 2, 5)
    assert np.abs(y - ref).sum() / np.abs(ref).sum() < 1e-4


@pytest.mark.parametrize("m,r", [(2, 3), (4, 3), (6, 3), (3, 5)])
def test_layer_1d_bitwise_vs_oracle(wino, orc, m, r):
    import torch
    x, w = inputs.layer_uniform(3, 7, 5, 1, 29, r=r, seed=11, dim=1)
    pts = [0.0, -1.5, 1.5, -1 / 1.5, 1 / 1.5, -1.0, 1.0, 2.5][: m + r - 2] + [math.inf]
    pad = 1
    y = torch.full((3, 5, 29 + 2 * pad - r + 1), float("nan"), device="cuda")
    wino.wino_conv1d(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(), y, pts, m, r, pad)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), orc.wino_layer(x, w, 1, pad, pts, m, r))


def test_layer_degenerate_inputs(wino):
    import torch
    x = torch.zeros((0, 4, 8, 8), device="cuda")
    w = torch.zeros((4, 4, 3, 3), device="cuda")
    y = torch.zeros((0, 4, 8, 8), device="cuda")
    wino.wino_conv2d(x, w, y, LAVIN, 2, 3, 1)  # N = 0: nothing to do
    with pytest.raises(wino.WinoError) as e:
        wino.wino_conv2d(torch.zeros((1, 4, 8, 8), device="cuda"), w,
                         torch.zeros((1, 4, 8, 8), device="cuda"), [0.0, 1.0, 1.0, math.inf], 2, 3)
    assert e.value.status == wino.WINO_ESINGULAR


@pytest.mark.parametrize("dim", [1, 2])
def test_direct_f64_vs_oracle(wino, orc, dim):
    import torch
    if dim == 2:
        x, w = inputs.layer_uniform(2, 6, 5, 13, 11, seed=3)
    else:
        x, w = inputs.layer_uniform(2, 6, 5, 1, 40, seed=3, dim=1)
    ref = orc.direct_f64(x, w, dim, 1, 3)
    y64 = torch.zeros(ref.shape, dtype=torch.float64, device="cuda")
    wino.wino_direct_conv_f64(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(), y64, 1)
    torch.cuda.synchronize()
    got = y64.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def _fused_launches(wino, fn):
    wino.wino_profile_enable(True)
    wino.wino_profile_read("fused_layer")
    try:
        fn()
    finally:
        wino.wino_profile_enable(False)
    return wino.wino_profile_read("fused_layer")[1]


# split tile shapes per m: single-CTA shapes, then (m = 4: split3-6, m = 6:
# split3-5) the cluster shapes whose CTAs split the frequencies
SPLIT_SHAPES = {2: 1, 4: 7, 6: 6}
VARIANTS = ["fused", "split"] + [f"split{c}" for c in range(1, 7)]


def _has_variant(m, variant):
    return not variant.startswith("split") or int(variant[5:] or 0) < SPLIT_SHAPES[m]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m", [2, 4, 6])
@pytest.mark.parametrize("shape", [(1, 13, 64, 17, 19, 1), (2, 70, 128, 9, 10, 1),
                                   (1, 3, 192, 6, 30, 0), (1, 9, 64, 1, 1, 2)])
def test_fused_layer_bitwise_vs_oracle(wino, orc, m, shape, variant, monkeypatch):
    """The fused kernel and the split transform + GEMM/output kernels in each
    tile shape (the cluster shapes included) on ragged tile blocks, channel
    counts off their chunking, several k-blocks, 1x1 images with padding."""
    if not _has_variant(m, variant):
        pytest.skip(f"F({m}x{m},3x3) has {SPLIT_SHAPES[m]} split tile shapes")
    monkeypatch.setenv("WINO_LAYER_VARIANT", variant)
    N, C, K, H, W, pad = shape
    x, w = inputs.layer_uniform(N, C, K, H, W, seed=100 + m)
    out = {}
    n = _fused_launches(wino, lambda: out.setdefault("y", _run2d(wino, x, w, POINTS[m], m, pad)))
    assert n == 1, "fused kernel not taken"
    assert np.array_equal(out["y"], orc.wino_layer(x, w, 2, pad, POINTS[m], m, 3))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m", [2, 4, 6])
@pytest.mark.parametrize("shape", [(2, 11, 64, 13, 16, 1), (1, 5, 64, 7, 22, 1),
                                   (3, 8, 64, 9, 36, 1)])
def test_row_vector_patches_bitwise_vs_oracle(wino, orc, m, shape, variant, monkeypatch):
    """Padding 1 and an even width: the input transforms load each patch
    row's interior columns as vectors and take the halo columns from the
    neighbouring lanes.  Widths a multiple of 4 and 2 mod 4, tile rows and
    columns cut by the image edge, tile blocks that start inside a tile row
    and channel counts off the chunking, in every tile shape: the same bits
    as the oracle."""
    if not _has_variant(m, variant):
        pytest.skip(f"F({m}x{m},3x3) has {SPLIT_SHAPES[m]} split tile shapes")
    monkeypatch.setenv("WINO_LAYER_VARIANT", variant)
    N, C, K, H, W, pad = shape
    x, w = inputs.layer_uniform(N, C, K, H, W, seed=300 + m)
    out = {}
    n = _fused_launches(wino, lambda: out.setdefault("y", _run2d(wino, x, w, POINTS[m], m, pad)))
    assert n == 1, "fused kernel not taken"
    assert np.array_equal(out["y"], orc.wino_layer(x, w, 2, pad, POINTS[m], m, 3))


@pytest.mark.slow
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m", [4, 6])
@pytest.mark.parametrize("layer", [0, 3])
def test_vgg_full_size_sampled_tiles(wino, orc, m, layer, variant, monkeypatch):
    """The bench's configuration (VGG16 stage, N = 32, the bench's points):
    512 random (tile, k) pairs recomputed by the oracle match bit for bit."""
    import torch
    if not _has_variant(m, variant):
        pytest.skip(f"F({m}x{m},3x3) has {SPLIT_SHAPES[m]} split tile shapes")
    monkeypatch.setenv("WINO_LAYER_VARIANT", variant)
    C, H = inputs.VGG16_LAYERS[layer]
    x, w = inputs.vgg_layer_host(C, H, N=inputs.VGG_BATCH, seed=7)
    pts = POINTS[4] if m == 4 else [0.0, -0.5, -2.0, 2.0, 0.5, -1.003, 1.003, math.inf]
    y = torch.empty((inputs.VGG_BATCH, C, H, H), device="cuda")
    xt, wt = torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda()
    n = _fused_launches(wino, lambda: wino.wino_conv2d(xt, wt, y, pts, m, 3, 1))
    assert n == 1
    yh = y.cpu().numpy()
    th = -(-H // m)
    T = inputs.VGG_BATCH * th * th
    rng = np.random.default_rng(layer * 10 + m)
    sel = np.stack([rng.integers(0, T, 512), rng.integers(0, C, 512)], axis=1)
    out = orc.wino_layer_tiles(x, w, 2, 1, pts, m, 3, sel)
    for (t, k), o in zip(sel, out):
        nn, ti, tj = t // (th * th), (t // th) % th, t % th
        for a in range(m):
            for b in range(m):
                p, q = ti * m + a, tj * m + b
                if p < H and q < H:
                    assert o[a, b] == yh[nn, k, p, q], (t, k, a, b)


def test_error_stats_vs_numpy(wino):
    import torch
    rng = np.random.default_rng(5)
    y = rng.normal(0, 1, 1_000_003)
    yh = (y + rng.normal(0, 1e-6, y.size)).astype(np.float32)
    got = wino.wino_error_stats(torch.from_numpy(yh).cuda(), torch.from_numpy(y).cuda())
    e = np.abs(yh.astype(np.float64) - y)
    want = (e.sum(), np.abs(y).sum(), e.max(), np.abs(y).max())
    for a, b in zip(got, want):
        assert a == pytest.approx(b, rel=1e-12)
    # a NaN output is not hidden behind the largest finite error
    yh[12345] = np.nan
    got = wino.wino_error_stats(torch.from_numpy(yh).cuda(), torch.from_numpy(y).cuda())
    assert np.isnan(got[0]) and np.isnan(got[2]) and got[3] == pytest.approx(want[3], rel=1e-12)


def test_no_bounded_wait_gave_up(wino, monkeypatch):
    """Every layer form (each FP32 split tile shape, single-CTA and cluster,
    with their bulk copies; the fused kernel; the tensor-core forms)
    completed its waits: the device's wait-error flag is clear."""
    import torch
    wino.wino_wait_error()
    x, w = inputs.layer_uniform(2, 70, 128, 9, 10, seed=3)
    xt, wt = torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda()
    y = torch.empty((2, 128, 9, 10), device="cuda")
    for m in (4, 6):
        for v in [v for v in VARIANTS if _has_variant(m, v)]:
            monkeypatch.setenv("WINO_LAYER_VARIANT", v)
            wino.wino_conv2d(xt, wt, y, POINTS[m], m, 3, 1)
    monkeypatch.delenv("WINO_LAYER_VARIANT")
    for dt in ("bf16", "split_bf16x6"):
        wino.wino_conv2d(xt, wt, y, POINTS[4], 4, 3, 1, dt)
    assert not wino.wino_wait_error()


def test_bounded_wait_gives_up_and_reports(wino):
    """The give-up path of the layer kernels' bounded waits, run on purpose:
    a wait on an mbarrier that nothing arrives at ends after its poll limit,
    the kernel returns, the device flag reads set once and is then clear,
    and the device stays usable."""
    import torch
    wino.wino_wait_error()
    ns = wino.wino_wait_probe(256)
    assert ns > 0
    assert wino.wino_wait_error()
    assert not wino.wino_wait_error()
    # the context is intact: a layer still runs and matches the oracle
    x, w = inputs.layer_uniform(1, 13, 64, 17, 19, seed=5)
    y = torch.empty((1, 64, 17, 19), device="cuda")
    wino.wino_conv2d(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(), y, POINTS[4], 4, 3,
                     1)
    assert np.all(np.isfinite(y.cpu().numpy()))
    assert not wino.wino_wait_error()
    # the layer kernels' limit at the measured time per failed poll: a wait
    # that can never complete is abandoned within a few seconds
    import pathlib
    import re
    hdr = (pathlib.Path(__file__).resolve().parents[1] / "include" / "wino.h").read_text()
    polls = 1 << int(re.search(r"#define WINO_WAIT_POLLS \(1 << (\d+)\)", hdr).group(1))
    assert ns / 256 * polls < 5e9, (ns / 256, polls)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "split_bf16x6"])
def test_layer_on_a_caller_stream(wino, dtype):
    """A layer call enqueues part of its work (the filter transforms) on the
    library's side stream and joins it back to the caller's stream: a caller
    who waits for their own stream only sees the finished output, the same
    bits as a call on the default stream.  The caller's stream starts behind
    a long kernel, so the side stream's work would run ahead of it unless
    the fork orders it."""
    import torch
    C, H, N = 128, 56, 8
    x, w = inputs.vgg_layer_device(C, H, N=N, seed=3)
    y0 = torch.empty((N, C, H, H), device="cuda")
    wino.wino_conv2d(x, w, y0, POINTS[4], 4, 3, 1, dtype)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    y1 = torch.full_like(y0, float("nan"))
    w1 = torch.zeros_like(w)
    with torch.cuda.stream(s):
        torch.cuda._sleep(20_000_000)  # the caller's stream is busy ...
        w1.copy_(w)                    # ... and only then holds the weights
        wino.wino_conv2d(x, w1, y1, POINTS[4], 4, 3, 1, dtype, stream=s)
    s.synchronize()
    assert torch.equal(y1, y0)
