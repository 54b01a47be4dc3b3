"""GPU parity of the summation-order variants of the sweep (Sec. 5: the
Huffman order the paper's tables use, alone and with FP64 transforms)
against the oracle: explicit point sets at every compiled size, the mask
sweep on a c sample, its top-10 c ranking, and the agreement of the two
front ends."""
import math

import numpy as np
import pytest

from paper_2201_10369_gb300 import inputs
from paper_2201_10369_gb300.inputs import COMPARISON_SETS, PROPOSED_SETS, chebyshev_points

pytestmark = pytest.mark.gpu

INF = math.inf
REL = 1e-6
ORDERS = ["huffman", "huffman_mixed"]
GPU_N = [(1, n) for n in range(4, 11)] + [(2, n) for n in range(4, 11)]


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("dim,n", GPU_N)
def test_order_pointsets_vs_oracle(wino, orc, order, dim, n):
    m = n - 2
    sets = [COMPARISON_SETS[(dim, n)] + [INF], PROPOSED_SETS[(dim, n)] + [INF],
            chebyshev_points(n - 1) + [INF]]
    got = wino.wino_pointset_error((dim, m, 3), sets, 1000, seed=2, order=order)
    want = orc.pointset_error_order(dim, m, 3, sets, 1000, 2, order)
    assert np.all(np.abs(got - want) <= REL * want), (got, want)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("m", [2, 4, 6])
def test_order_r5_vs_oracle(wino, orc, order, m):
    """1D r = 5 (Table 1's 5-tap kernels) in both orders."""
    n = m + 4
    sets = [chebyshev_points(n - 1) + [INF], [0.0] + [s * k for k in (0.5, 1, 2, 3)
                                                      for s in (-1, 1)][:n - 2] + [INF]]
    got = wino.wino_pointset_error((1, m, 5), sets, 500, seed=3, order=order)
    want = orc.pointset_error_order(1, m, 5, sets, 500, 3, order)
    assert np.all(np.abs(got - want) <= REL * want), (got, want)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("size,masks", [((1, 4, 3, 1.0), [0x0F, 0x66, 0x63]),
                                        ((2, 4, 3, 1.0), [0x0F, 0x66]),
                                        ((2, 6, 3, 1.0), [0x6F]),
                                        ((1, 7, 3, 2.478), [0x7F, 0xF7])])
def test_order_mask_sweep_vs_oracle(wino, orc, order, size, masks):
    """The mask sweep against the oracle on the same point sets, on a c
    sample spread over the grid, and the top-10 c per mask identical."""
    dim, m, r, d = size
    cg = inputs.c_grid(4096)[::97]
    got = wino.wino_error_sweep(cg, [size], masks, 400, seed=1, order=order)[0]
    for qi, mk in enumerate(masks):
        sets = [orc.mask_points(dim, m, r, d, mk, c) for c in cg]
        want = orc.pointset_error_order(dim, m, r, sets, 400, 1, order)
        fin = np.isfinite(want)
        assert np.array_equal(np.isfinite(got[qi]), fin)
        assert np.all(np.abs(got[qi][fin] - want[fin]) <= REL * want[fin])
        top_g = np.lexsort((np.arange(cg.size), got[qi]))[:10]
        top_w = np.lexsort((np.arange(cg.size), want))[:10]
        assert np.array_equal(top_g, top_w)


@pytest.mark.parametrize("order", ORDERS)
def test_order_pointset_same_bits_as_mask_sweep(wino, order):
    """P8 is the full c-group at c = 2, d = 1 (mask 0x6f): both front ends
    build the same instance and return the same bits."""
    p8 = [[0.0, -1.0, 1.0, 0.5, -0.5, 2.0, -2.0, INF]]
    for dim in (1, 2):
        a = wino.wino_pointset_error((dim, 6, 3), p8, 300, seed=4, order=order)[0]
        b = wino.wino_error_sweep([2.0], [(dim, 6, 3, 1.0)], [0x6F], 300, seed=4,
                                  order=order)[0, 0, 0]
        assert a == b


def test_order_fma_is_the_plain_sweep(wino):
    """WINO_ORDER_FMA through the order entry points is the plain sweep."""
    import ctypes
    L = wino.load()
    cg = np.ascontiguousarray(inputs.c_grid(64))
    sz = (wino.WinoSize * 1)(wino.WinoSize(2, 4, 3, 1.0))
    mk = (ctypes.c_ubyte * 1)(0x0F)
    e = np.empty(64)
    dp = ctypes.POINTER(ctypes.c_double)
    assert L.wino_error_sweep_order(cg.ctypes.data_as(dp), 64, sz, 1, mk, 1, 200, 0,
                                    wino.WINO_ORDER_FMA, e.ctypes.data_as(dp), None) == 0
    assert np.array_equal(e, wino.wino_error_sweep(cg, [(2, 4, 3, 1.0)], [0x0F], 200)[0, 0])


@pytest.mark.parametrize("order", ORDERS)
def test_order_degenerate_sets(wino, order):
    e = wino.wino_pointset_error((1, 2, 3), [[0.0, 1.0, 1.0, INF], [0.0, 1.0, -1.0, INF]], 64,
                                 order=order)
    assert e[0] == INF and np.isfinite(e[1])


def test_order_moves_the_error_by_percents(wino):
    """Across the sweep's sizes the Huffman order stays within a factor 1.5 of
    the plain order and the FP64 transforms lower the error (Sec. 5)."""
    for size, mk in [((1, 6, 3, 1.0), 0x6F), ((2, 4, 3, 1.0), 0x0F), ((2, 6, 3, 1.0), 0x6F)]:
        cg = inputs.c_grid(256)
        e = {o: wino.wino_error_sweep(cg, [size], [mk], 500, order=o)[0, 0]
             for o in ("fma", "huffman", "huffman_mixed")}
        ok = np.isfinite(e["fma"])
        ratio = np.median(e["huffman"][ok] / e["fma"][ok])
        assert 1 / 1.5 < ratio < 1.5, (size, ratio)
        assert np.median(e["huffman_mixed"][ok] / e["huffman"][ok]) < 1.0


@pytest.mark.parametrize("order", ["fma"] + ORDERS)
def test_order_mask_sweep_matches_pointsets_every_size(wino, orc, order):
    """Every compiled size: the mask sweep's errors for the first valid mask
    at a few c equal, bit for bit, the point-set errors of the same sets
    (both front ends, same trials and summation order)."""
    cg = inputs.c_grid(4096)[::601]
    masks = inputs.sweep_masks()
    for size in (inputs.SWEEP_SIZES + [(1, m, 5, 2.0) for m in range(2, 7)]
                 + [(2, m, 5, 2.0) for m in range(2, 5)] + [(2, 7, 3, 2.485), (2, 8, 3, 2.099)]):
        dim, m, r, d = size
        mk = wino.valid_masks(size, masks)[0]
        e = wino.wino_error_sweep(cg, [size], [mk], 256, seed=5, order=order)[0, 0]
        sets = [orc.mask_points(dim, m, r, d, mk, c) for c in cg]
        p = wino.wino_pointset_error((dim, m, r), sets, 256, seed=5, order=order)
        assert np.all(np.isfinite(e)), (size, order)
        assert np.array_equal(e, p), (size, order, e, p)
