"""GPU parity of the precision form of the contraction (tcgen05 BF16 / FP16 /
split BF16x3 / split BF16x6 with per-frequency power-of-two scaling) against
the oracle's emulation of the same rounding.

Both sides round the same FP32 transform outputs to the same 16-bit
operands and form exact products (16-bit x 16-bit products fit FP32).  They
differ only in how the FP32 accumulator sums those products over the
channels: the oracle adds them one after the other with fmaf, the tensor
cores in their own order, with an adder whose rounding is not documented.
The bar is derived from that (reading in the design notes):
  - a sum of n exact terms p_i in FP32 errs by at most gamma_n(v) sum |p_i|,
    gamma_n(v) = n v / (1 - n v), with v = 2^-24 for the oracle's
    round-to-nearest and v = 2^-23 for the tensor cores (any rounding that
    errs by at most one unit in the last place, truncation included);
  - n = (products per channel) x C (+ 1 for split BF16x6, whose two
    accumulators are added once at the end), and sum |p_i| <= 1.1 sum_c
    |U_c| |V_c| (the parts of an operand sum in magnitude to at most
    (1 + 2^-7) of it);
  - the output transform A^T M A maps the difference of M through |A^T| .
    |A| and rounds both sides' results, each by at most gamma_{2 alpha}(2^-24)
    |A^T| |M| |A| <= gamma_{2 alpha} |A^T| S |A|, S = sum_c |U| |V|.
So, per output: |y_gpu - y_oracle| <= (1.1 (gamma_n(2^-24) + gamma_n(2^-23))
+ 2 gamma_{2 alpha}(2^-24)) (|A^T| S |A|), with U, V and S computed here in
FP64 from the FP64 matrices.  The relative L1 errors against FP64 then
differ by at most sum(bound) / sum|y_fp64|.  Besides the derived bars: the
BF16 / FP16 / split BF16x3 errors, dominated by the operand rounding both
sides share, agree within 5%; and up to C = 128 the split BF16x6 error (its
operands exact, so the accumulation dominates) is no more than 1.05x the
sequential emulation's."""
import math

import numpy as np
import pytest

from paper_2201_10369_gb300 import inputs

pytestmark = pytest.mark.gpu

PTS = {4: [0.0, -1 / 1.622, -1.622, 1.622, 1 / 1.622, math.inf],
       6: [0.0, -0.5, -2.0, 2.0, 0.5, -1.003, 1.003, math.inf],
       2: [0.0, -1.0, 1.0, math.inf]}


PRODUCTS = {"bf16": 1, "fp16": 1, "split_bf16x3": 3, "split_bf16x6": 6}


def _gamma(n, v):
    return n * v / (1.0 - n * v)


def _patches(x, m, pad):
    """Input tiles d[n][ti][tj][c][alpha][alpha] (zero padding, ragged
    tiles zero-filled), FP64."""
    N, C, H, W = x.shape
    a = m + 2
    Ho, Wo = H + 2 * pad - 2, W + 2 * pad - 2
    th, tw = -(-Ho // m), -(-Wo // m)
    xp = np.zeros((N, C, th * m + 2, tw * m + 2))
    xp[:, :, pad:pad + H, pad:pad + W] = x
    d = np.empty((N, th, tw, C, a, a))
    for i in range(th):
        for j in range(tw):
            d[:, i, j] = xp[:, :, i * m:i * m + a, j * m:j * m + a]
    return d, th, tw


def tc_magnitudes(orc, x, w, pts, m):
    """|A^T| S |A| per output, S[f][t][k] = sum_c |U[f][t][c]| |V[f][c][k]|,
    U = B^T d B and V = G g G^T in FP64 from the FP64 matrices; shaped like
    y [N][K][Ho][Wo] (pad 1, r = 3)."""
    AT, G, BT = orc.make_matrices(pts, m, 3)
    N, C, H, W = x.shape
    K = w.shape[0]
    a = m + 2
    d, th, tw = _patches(x.astype(np.float64), m, 1)
    U = np.einsum("il,ntsclq,jq->ijntsc", BT, d, BT).reshape(a * a, N * th * tw, C)
    V = np.einsum("ip,kcpq,jq->ijck", G, w.astype(np.float64), G).reshape(a * a, C, K)
    S = np.matmul(np.abs(U), np.abs(V)).reshape(a, a, N, th, tw, K)
    Y = np.einsum("ai,ijntsk,bj->nktasb", np.abs(AT), S, np.abs(AT))
    return Y.reshape(N, K, th * m, tw * m)[:, :, :H, :W]


def tc_parity_bound(orc, x, w, pts, m, dtype):
    """Per-output bound on |y_gpu - y_oracle| (see the module docstring)."""
    a = m + 2
    n = PRODUCTS[dtype] * x.shape[1] + (1 if dtype == "split_bf16x6" else 0)
    f = 1.1 * (_gamma(n, 2.0 ** -24) + _gamma(n, 2.0 ** -23)) + 2 * _gamma(2 * a, 2.0 ** -24)
    return f * tc_magnitudes(orc, x, w, pts, m)


@pytest.mark.parametrize("dtype", ["bf16", "fp16", "split_bf16x3", "split_bf16x6"])
@pytest.mark.parametrize("m", [4, 6, 2])
@pytest.mark.parametrize("shape", [(2, 64, 64, 10, 10), (1, 80, 128, 9, 13), (1, 64, 256, 6, 6),
                                   (1, 300, 128, 7, 9), (1, 64, 64, 11, 24)])
def test_tc_layer_vs_oracle_emulation(wino, orc, dtype, m, shape):
    import torch
    N, C, K, H, W = shape
    rng = np.random.default_rng(C + K + m)
    x = np.maximum(rng.standard_normal((N, C, H, W)), 0).astype(np.float32)
    w = (rng.standard_normal((K, C, 3, 3)) * np.sqrt(2.0 / (9 * C))).astype(np.float32)
    y = torch.full((N, K, H, W), float("nan"), device="cuda")
    wino.wino_conv2d(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(), y, PTS[m], m, 3, 1,
                     dtype)
    torch.cuda.synchronize()
    yg = y.cpu().numpy()
    yo = orc.wino_layer(x, w, 2, 1, PTS[m], m, 3, dtype)
    assert np.all(np.isfinite(yg))
    bound = tc_parity_bound(orc, x, w, PTS[m], m, dtype)
    diff = np.abs(yg.astype(np.float64) - yo)
    assert np.all(diff <= bound), float((diff / bound).max())
    ref = orc.direct_f64(x, w, 2, 1, 3)
    sref = np.abs(ref).sum()
    eg = np.abs(yg - ref).sum() / sref
    eo = np.abs(yo.astype(np.float64) - ref).sum() / sref
    assert abs(eg - eo) <= bound.sum() / sref, (eg, eo, bound.sum() / sref)
    if dtype == "split_bf16x6":
        # operands exact to 2^-24: the accumulation is the dominant error
        # term, and over short contractions the tensor cores' is as good as
        # sequential FP32
        if C <= 128:
            assert eg <= 1.05 * eo, (eg, eo)
    else:
        assert abs(eg / eo - 1) < 0.05, (eg, eo)


@pytest.mark.parametrize("dtype", ["bf16", "fp16", "split_bf16x3", "split_bf16x6"])
@pytest.mark.parametrize("C", [64, 128, 300, 512])
def test_tc_exact_regime_every_chunk(wino, orc, dtype, C):
    """Integer inputs in [-2, 2] with F(2x2,3x3) on {0, 1, -1, inf}: every
    operand and partial sum is exact, so the result is the exact correlation
    whatever the accumulation order -- a chunk lost, repeated or read from the
    wrong stage of the multi-stage ring (C > 64) would show."""
    import torch
    rng = np.random.default_rng(C)
    x = rng.integers(-2, 3, (1, C, 10, 12)).astype(np.float32)
    w = rng.integers(-2, 3, (32, C, 3, 3)).astype(np.float32)
    y = torch.full((1, 32, 10, 12), float("nan"), device="cuda")
    wino.wino_conv2d(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(), y, PTS[2], 2, 3, 1,
                     dtype)
    torch.cuda.synchronize()
    ref = orc.direct_f64(x, w, 2, 1, 3)
    assert np.array_equal(y.cpu().numpy().astype(np.float64), ref)


def test_tc_error_ordering_matches_precision(wino, orc):
    """BF16 > FP16 > split BF16x3 > FP32 >= split BF16x6 in error against FP64
    (F(4x4,3x3))."""
    import torch
    x, w = inputs.vgg_layer_host(64, 20, N=2, seed=3)
    xt, wt = torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda()
    ref = orc.direct_f64(x, w, 2, 1, 3)
    err = {}
    for dt in ("f32", "bf16", "fp16", "split_bf16x3", "split_bf16x6"):
        y = torch.empty((2, 64, 20, 20), device="cuda")
        wino.wino_conv2d(xt, wt, y, PTS[4], 4, 3, 1, dt)
        torch.cuda.synchronize()
        err[dt] = np.abs(y.cpu().numpy() - ref).sum() / np.abs(ref).sum()
    assert err["bf16"] > err["fp16"] > err["split_bf16x3"] > err["f32"] >= err["split_bf16x6"]


def _sample_bound(orc, x, w, pts, m, sel, dtype):
    """The per-output bound of the module docstring for sampled (tile, k)
    pairs of a full layer: [n_sel][m][m]."""
    AT, G, BT = orc.make_matrices(pts, m, 3)
    N, C, H, W = x.shape
    a = m + 2
    th, tw = -(-H // m), -(-W // m)
    n_terms = PRODUCTS[dtype] * C + (1 if dtype == "split_bf16x6" else 0)
    fac = (1.1 * (_gamma(n_terms, 2.0 ** -24) + _gamma(n_terms, 2.0 ** -23))
           + 2 * _gamma(2 * a, 2.0 ** -24))
    out = np.empty((len(sel), m, m))
    for s, (t, k) in enumerate(sel):
        n, ti, tj = t // (th * tw), (t // tw) % th, t % tw
        d = np.zeros((C, a, a))
        h0, w0 = ti * m - 1, tj * m - 1
        hs, ws = max(h0, 0), max(w0, 0)
        he, we = min(h0 + a, H), min(w0 + a, W)
        d[:, hs - h0:he - h0, ws - w0:we - w0] = x[n, :, hs:he, ws:we]
        U = np.einsum("il,clq,jq->cij", BT, d, BT)
        V = np.einsum("ip,cpq,jq->cij", G, w[k].astype(np.float64), G)
        S = (np.abs(U) * np.abs(V)).sum(axis=0)
        out[s] = fac * (np.abs(AT) @ S @ np.abs(AT).T)
    return out


@pytest.mark.parametrize("layer", [0, 3])
def test_tc_vgg_full_size_sampled(wino, orc, layer):
    """The bench's configuration (VGG16 stage, N = 32, the bench's points)
    for every tensor-core dtype and both tile sizes: 256 random (tile, k)
    outputs recomputed by the oracle's emulation of the same rounding agree
    within the derived per-output bound."""
    import torch
    C, H = inputs.VGG16_LAYERS[layer]
    x, w = inputs.vgg_layer_host(C, H, N=inputs.VGG_BATCH, seed=5 + layer)
    xt, wt = torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda()
    y = torch.empty((inputs.VGG_BATCH, C, H, H), device="cuda")
    for m in (4, 6):
        th = -(-H // m)
        T = inputs.VGG_BATCH * th * th
        rng = np.random.default_rng(100 * layer + m)
        sel = np.stack([rng.integers(0, T, 256), rng.integers(0, C, 256)], axis=1)
        for dtype in PRODUCTS:
            y.fill_(float("nan"))
            wino.wino_conv2d(xt, wt, y, PTS[m], m, 3, 1, dtype)
            torch.cuda.synchronize()
            yh = y.cpu().numpy()
            out = orc.wino_layer_tiles(x, w, 2, 1, PTS[m], m, 3, sel, dtype)
            bound = _sample_bound(orc, x, w, PTS[m], m, sel, dtype)
            for s, (t, k) in enumerate(sel):
                nn, ti, tj = t // (th * th), (t // th) % th, t % th
                for a in range(m):
                    for b in range(m):
                        p, q = ti * m + a, tj * m + b
                        if p < H and q < H:
                            diff = abs(float(yh[nn, k, p, q]) - float(out[s, a, b]))
                            assert diff <= bound[s, a, b], (m, dtype, t, k, a, b, diff)
