"""The guided search, the random search and their host logic behind the C
ABI (wino_guided_*, wino_random_search), called through ctypes.

The planned sweep returns the same bits as wino_error_sweep for the same
(size, mask, c) (one summation order for every path), so every result of a
search must be exactly the exhaustive sweep's error at the c it reports:
that checks the searches' argmin, index and grid bookkeeping bit for bit,
whatever the network predicts."""
import ctypes

import numpy as np
import pytest

from paper_2201_10369_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [(1, 2, 3, 1.0), (1, 3, 3, 1.0), (1, 4, 3, 1.0), (2, 2, 3, 1.0)]
TRIALS = 200


def _abi_guided(wino, model, sizes, masks, cg, top, probe, refine, guard, seed=5):
    """wino_guided_create / run / destroy, called directly."""
    import torch
    L = wino.load()
    cg = np.ascontiguousarray(cg, dtype=np.float64)
    mk = np.ascontiguousarray(masks, dtype=np.uint8)
    sz = (wino.WinoSize * len(sizes))(*[wino.WinoSize(*s) for s in sizes])
    prm = wino.WinoGuidedParams(top, probe, refine, guard)
    h = ctypes.c_void_p()
    UB = ctypes.POINTER(ctypes.c_ubyte)
    assert L.wino_guided_create(model._h, sz, len(sizes), mk.ctypes.data_as(UB), mk.size,
                                cg.ctypes.data_as(wino._DP), cg.size, TRIALS, seed,
                                ctypes.byref(prm), ctypes.byref(h)) == wino.WINO_OK, \
        wino.wino_last_error()
    try:
        best = np.empty((len(sizes), mk.size))
        best_c = np.empty_like(best)
        st = wino.WinoGuidedStats()
        assert L.wino_guided_run(h, best.ctypes.data_as(wino._DP), best_c.ctypes.data_as(wino._DP),
                                 ctypes.byref(st),
                                 torch.cuda.current_stream().cuda_stream) == wino.WINO_OK
    finally:
        L.wino_guided_destroy(h)
    return best, best_c, st


@pytest.fixture(scope="module")
def setup(wino):
    masks = inputs.sweep_masks()
    cg = inputs.c_grid(512)
    ex = wino.wino_error_sweep(cg, SIZES, masks, TRIALS, seed=5)
    model = wino.Surrogate(seed=1)
    rng = np.random.default_rng(2)
    model.set_params(rng.normal(0, 0.3, wino.MLP_PARAMS).astype(np.float32))
    yield masks, cg, ex, model
    model.close()


def _check_results_are_grid_values(ex, best, best_c, cg):
    valid = np.any(np.isfinite(ex), axis=2)
    assert np.array_equal(np.isfinite(best), valid)
    for s, q in zip(*np.nonzero(valid)):
        k = int(np.nonzero(cg == best_c[s, q])[0][0])
        assert best[s, q] == ex[s, q, k]                       # exactly a grid value
        assert best[s, q] >= np.nanmin(np.where(np.isinf(ex[s, q]), np.nan, ex[s, q]))
    return valid


@pytest.mark.parametrize("guard", [1.01, 1.0])
def test_guided_search_host_logic(wino, setup, guard):
    masks, cg, ex, model = setup
    top, probe, refine = 16, 16, 8
    best, best_c, st = _abi_guided(wino, model, SIZES, masks, cg, top, probe, refine, guard)
    valid = _check_results_are_grid_values(ex, best, best_c, cg)
    assert st.rows == int(valid.sum())
    assert st.evaluated == st.rows * (top + probe + 2 * refine + 1) + st.fallback_rows * cg.size
    assert 0 <= st.fallback_rows <= st.rows


def test_guided_search_whole_grid_proposed_finds_every_row_minimum(wino, setup):
    """top = n_c: the network proposes every grid point, so its region holds
    the row minimum, no row can fall back and every result is the minimum."""
    masks, cg, ex, model = setup
    best, best_c, st = _abi_guided(wino, model, SIZES, masks, cg, cg.size, 4, 2, 1.01)
    valid = _check_results_are_grid_values(ex, best, best_c, cg)
    exf = np.where(np.isfinite(ex), ex, np.inf)
    assert st.fallback_rows == 0
    assert np.array_equal(best[valid], exf.min(axis=2)[valid])


def test_random_search_results_are_grid_values(wino, setup):
    masks, cg, ex, _ = setup
    best = wino.random_search(SIZES, masks, cg, TRIALS, 32, seed=5)
    valid = np.any(np.isfinite(ex), axis=2)
    assert np.array_equal(np.isfinite(best), valid)
    for s, q in zip(*np.nonzero(valid)):
        assert best[s, q] in set(ex[s, q][np.isfinite(ex[s, q])].tolist())
    # the whole grid as the budget with a huge draw count finds the minimum
    big = wino.random_search(SIZES, masks, cg, TRIALS, 16 * cg.size, seed=5)
    exf = np.where(np.isfinite(ex), ex, np.inf)
    assert np.array_equal(big[valid], exf.min(axis=2)[valid])


def test_guided_create_validation(wino, setup):
    masks, cg, _, model = setup
    L = wino.load()
    h = ctypes.c_void_p()
    sz = (wino.WinoSize * 1)(wino.WinoSize(1, 2, 3, 1.0))
    mk = np.ascontiguousarray(masks, dtype=np.uint8)
    UB = ctypes.POINTER(ctypes.c_ubyte)
    for prm in (wino.WinoGuidedParams(0, 4, 2, 1.01), wino.WinoGuidedParams(4, 4, 2, 0.9),
                wino.WinoGuidedParams(cg.size + 1, 4, 2, 1.01)):
        assert L.wino_guided_create(model._h, sz, 1, mk.ctypes.data_as(UB), mk.size,
                                    cg.ctypes.data_as(wino._DP), cg.size, TRIALS, 0,
                                    ctypes.byref(prm), ctypes.byref(h)) == wino.WINO_EINVAL
