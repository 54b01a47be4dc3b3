"""GPU parity of the point sweep (wino_error_sweep) and of its device FP64
matrix construction (wino_instance_matrices) against the CPU oracle.

Bars: matrices 1e-13 relative; per-instance error 1e-6 relative (the GPU
reduces |yhat - y| per trial in FP32 with y split into two FP32 words, the
oracle in FP64; the parity bar is 3%); NaN / +inf positions identical; the
top-10 c ranking of each (size, mask) identical up to near-ties (oracle
errors within 1e-6 relative may swap)."""
import math

import numpy as np
import pytest

from paper_2201_10369_gb300 import inputs

pytestmark = pytest.mark.gpu

REL = 1e-6


@pytest.mark.parametrize("size,mask", [((1, 4, 3, 1.0), 0x0F), ((2, 6, 3, 1.0), 0x6F),
                                       ((1, 8, 3, 1.229), 0xFF), ((1, 4, 5, 1.0), 0x6F),
                                       ((2, 2, 3, 1.0), 0x28), ((1, 7, 3, 2.478), 0x7F)])
def test_instance_matrices_vs_oracle(wino, orc, size, mask):
    cg = np.concatenate([inputs.c_grid(256), [1.0, 2.0, 0.5]])
    AT, G, BT, sing = wino.wino_instance_matrices(cg, size, mask)
    dim, m, r, d = size
    for k, c in enumerate(cg):
        pts = orc.mask_points(dim, m, r, d, mask, c)
        try:
            want = orc.make_matrices(pts, m, r)
        except orc.SingularPoints:
            assert sing[k]
            continue
        assert not sing[k]
        for got, ref in zip((AT[k], G[k], BT[k]), want):
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def _top10_consistent(eg, eo):
    n = eo.size
    idx = np.arange(n)
    fin = np.isfinite(eo)
    oo = np.lexsort((idx[fin], eo[fin]))[:10]
    og = np.lexsort((idx[fin], eg[fin]))[:10]
    io, ig = idx[fin][oo], idx[fin][og]
    vo, vg = eo[io], eo[ig]
    assert np.all(np.abs(vg - vo) <= REL * np.abs(vo)), (io, ig)
    return int(np.sum(io == ig))


def test_sweep_small_grid_vs_oracle(wino, orc):
    """All 12 sizes x the 66 visited subsets, 48 c values (c = 1 included:
    coinciding points for many masks), 300 trials."""
    cg = np.sort(np.concatenate([inputs.c_grid(47), [1.0]]))
    sizes = inputs.SWEEP_SIZES
    masks = inputs.sweep_masks()
    eg = wino.wino_error_sweep(cg, sizes, masks, 300, seed=0)
    eo = orc.error_sweep(cg, sizes, masks, 300, 0, n_threads=8)
    assert np.array_equal(np.isnan(eg), np.isnan(eo))
    assert np.array_equal(np.isinf(eg), np.isinf(eo))
    fin = np.isfinite(eo)
    assert fin.sum() == 123 * 48 - np.isinf(eo).sum()
    assert np.all(np.abs(eg[fin] - eo[fin]) <= REL * eo[fin])
    exact = 0
    for s in range(len(sizes)):
        for q in range(masks.size):
            if np.isfinite(eo[s, q]).any():
                exact += _top10_consistent(eg[s, q], eo[s, q])
    assert exact >= 0.99 * 123 * 10


@pytest.mark.parametrize("m", [2, 3, 4])
def test_sweep_2d_r5_vs_oracle(wino, orc, m):
    """2D F(m x m, 5 x 5) (the 5x5 column of Table 1) in the sweep: every
    valid mask of the 66 with d = 2, 32 c values, 300 trials, against the
    oracle; the same top-10 c per mask."""
    cg = inputs.c_grid(4096)[::128]
    size = (2, m, 5, 2.0)
    masks = np.array(wino.valid_masks(size, inputs.sweep_masks()), np.uint8)
    eg = wino.wino_error_sweep(cg, [size], masks, 300, seed=1)[0]
    eo = orc.error_sweep(cg, [size], masks, 300, 1, n_threads=8)[0]
    assert np.array_equal(np.isinf(eg), np.isinf(eo))
    fin = np.isfinite(eo)
    assert fin.sum() > 0.9 * eo.size
    assert np.all(np.abs(eg[fin] - eo[fin]) <= REL * eo[fin])
    for q in range(masks.size):
        assert _top10_consistent(eg[q], eo[q]) >= 9


@pytest.mark.parametrize("size", [(2, 7, 3, 2.485), (2, 8, 3, 2.099)])
def test_sweep_wide_2d_vs_oracle(wino, orc, size):
    """2D F(7x7,3x3) and F(8x8,3x3) (Table 8, n = 9, 10), swept one warp per
    instance: every valid mask of the 66 at the paper's d, 24 c values, 200
    trials, against the oracle; the same top-10 c per mask."""
    cg = inputs.c_grid(4096)[::171]
    masks = np.array(wino.valid_masks(size, inputs.sweep_masks()), np.uint8)
    assert masks.size > 0
    eg = wino.wino_error_sweep(cg, [size], masks, 200, seed=2)[0]
    eo = orc.error_sweep(cg, [size], masks, 200, 2, n_threads=8)[0]
    assert np.array_equal(np.isinf(eg), np.isinf(eo))
    fin = np.isfinite(eo)
    assert fin.sum() > 0.9 * eo.size
    assert np.all(np.abs(eg[fin] - eo[fin]) <= REL * eo[fin])
    for q in range(masks.size):
        assert _top10_consistent(eg[q], eo[q]) >= 9


def test_sweep_seed_and_trials_change_results(wino):
    cg = inputs.c_grid(32)
    a = wino.wino_error_sweep(cg, [(2, 4, 3, 1.0)], [0x0F], 100, seed=0)
    b = wino.wino_error_sweep(cg, [(2, 4, 3, 1.0)], [0x0F], 100, seed=1)
    c = wino.wino_error_sweep(cg, [(2, 4, 3, 1.0)], [0x0F], 100, seed=0)
    assert np.array_equal(a, c) and not np.array_equal(a, b)


@pytest.mark.slow
def test_full_config_sweep_sampled(wino, orc):
    """The full sweep (4096 c x 1000 trials, 503 808 instances) on the GPU;
    the oracle recomputes 3 whole (size, mask) rows (top-10 ranking) and 40
    random instances one by one."""
    cg = inputs.c_grid()
    sizes = inputs.SWEEP_SIZES
    masks = inputs.sweep_masks()
    eg = wino.wino_error_sweep(cg, sizes, masks, inputs.SWEEP_TRIALS, seed=0)
    assert np.isfinite(eg).sum() + np.isinf(eg).sum() == 503808
    rows = [(2, 0x0F), (9, 0x0F), (7, 0x28)]  # 1D F(4,3), 2D F(4x4,3x3), 2D F(2x2,3x3)
    mlist = list(masks)
    for s, mk in rows:
        q = mlist.index(mk)
        eo = orc.error_sweep(cg, [sizes[s]], [mk], inputs.SWEEP_TRIALS, 0, n_threads=16)[0, 0]
        fin = np.isfinite(eo)
        assert np.all(np.abs(eg[s, q][fin] - eo[fin]) <= REL * eo[fin])
        assert _top10_consistent(eg[s, q], eo) >= 9
    rng = np.random.default_rng(0)
    valid = np.argwhere(np.isfinite(eg))
    for s, q, k in valid[rng.choice(len(valid), 40, replace=False)]:
        eo = orc.error_sweep([cg[k]], [sizes[s]], [masks[q]], inputs.SWEEP_TRIALS, 0)[0, 0, 0]
        assert abs(eg[s, q, k] - eo) <= REL * eo
