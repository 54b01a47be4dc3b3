"""GPU parity of the explicit point-set metric (the comparison sets of
Tables 7-8 and Chebyshev nodes) against the oracle, its agreement with the
mask sweep, and the paper's comparison: the best subset set of the proposed
family found by the exhaustive sweep against Barabasz's set of each size."""
import math

import numpy as np
import pytest

from paper_2201_10369_gb300 import inputs
from paper_2201_10369_gb300.inputs import (COMPARISON_SETS, PAPER_IMPROVEMENT_PCT, PROPOSED_SETS,
                                           chebyshev_points)

pytestmark = pytest.mark.gpu

INF = math.inf
REL = 1e-6
# sizes the GPU sweep is compiled for: (dim, n) with n = m + 2 points
GPU_N = [(1, n) for n in range(4, 11)] + [(2, n) for n in range(4, 11)]


@pytest.mark.parametrize("dim,n", GPU_N)
def test_pointsets_vs_oracle(wino, orc, dim, n):
    m = n - 2
    sets = [COMPARISON_SETS[(dim, n)] + [INF], PROPOSED_SETS[(dim, n)] + [INF],
            chebyshev_points(n - 1) + [INF]]
    got = wino.wino_pointset_error((dim, m, 3), sets, 1000, seed=2)
    want = orc.pointset_error(dim, m, 3, sets, 1000, 2)
    assert np.all(np.abs(got - want) <= REL * want), (got, want)


def test_pointset_same_bits_as_mask_sweep(wino):
    """P8 is the full c-group at c = 2, d = 1 (mask 0x6f): the same matrices on
    the same trials in the same summation order."""
    p8 = [[0.0, -1.0, 1.0, 0.5, -0.5, 2.0, -2.0, INF]]
    for dim in (1, 2):
        a = wino.wino_pointset_error((dim, 6, 3), p8, 300, seed=4)[0]
        b = wino.wino_error_sweep([2.0], [(dim, 6, 3, 1.0)], [0x6F], 300, seed=4)[0, 0, 0]
        assert a == b


def test_pointset_degenerate_and_unsupported(wino):
    e = wino.wino_pointset_error((1, 2, 3), [[0.0, 1.0, 1.0, INF], [0.0, 1.0, -1.0, INF]], 64)
    assert math.isinf(e[0]) and math.isfinite(e[1])
    with pytest.raises(wino.WinoError) as ex:
        wino.wino_pointset_error((1, 2, 3), [[0.0, 1.0, -1.0, 2.0]], 64)
    assert ex.value.status == wino.WINO_EINVAL
    with pytest.raises(wino.WinoError) as ex:  # 2D 7x7 kernels: not compiled
        wino.wino_pointset_error((2, 3, 7), [COMPARISON_SETS[(2, 9)] + [INF]], 64)
    assert ex.value.status == wino.WINO_EUNSUPPORTED


def test_paper_comparison(wino):
    """Tables 7-8 on the GPU: (1) the paper's proposed set against Barabasz's
    set reproduces the printed improvement's sign where it exceeds 5%
    (SIGN_EXCEPTIONS aside); (2) the exhaustive sweep of the proposed family
    (every subset, the 4096-value c grid, the paper's d for F(7,3), F(8,3))
    finds a set at least as good as Barabasz's at every size -- also at
    n = 7, where the paper's own pick lost by 13-14%."""
    from test_oracle_pointsets import SIGN_EXCEPTIONS
    cg = inputs.c_grid()
    masks = inputs.sweep_masks()
    sizes = {s[:2]: s for s in inputs.SWEEP_SIZES}
    # the wide 2D sizes at the paper's d (Table 8, n = 9, 10)
    sizes[(2, 7)] = (2, 7, 3, 2.485)
    sizes[(2, 8)] = (2, 8, 3, 2.099)
    for dim, n in GPU_N:
        m = n - 2
        pn, prop = wino.wino_pointset_error(
            (dim, m, 3), [COMPARISON_SETS[(dim, n)] + [INF], PROPOSED_SETS[(dim, n)] + [INF]], 1000)
        paper = PAPER_IMPROVEMENT_PCT[(dim, n)]
        if abs(paper) > 5.0 and (dim, n) not in SIGN_EXCEPTIONS:
            assert np.sign(pn - prop) == np.sign(paper), (dim, n, pn, prop, paper)
        ex = wino.wino_error_sweep(cg, [sizes[(dim, m)]], masks, 1000, seed=0)[0]
        best = np.nanmin(np.where(np.isinf(ex), np.nan, ex))
        assert best <= pn, (dim, n, best, pn)


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
@pytest.mark.parametrize("pairwise", [False, True])
def test_kron_form_vs_oracle(wino, orc, n, pairwise):
    """The Kronecker-product 2D form (Sec. 7) on the GPU against the oracle."""
    m = n - 2
    sets = [COMPARISON_SETS[(2, n)] + [INF], PROPOSED_SETS[(2, n)] + [INF]]
    got = wino.wino_pointset_error_kron(m, sets, 1000, seed=2, pairwise=pairwise)
    want = orc.pointset_error_kron(m, 3, sets, 1000, 2, pairwise)
    assert np.all(np.abs(got - want) <= REL * want), (got, want)


def test_kron_form_larger_error_on_gpu(wino):
    """Sec. 7's finding on the GPU: the Kronecker-product form and its pairwise
    variant give larger errors than the nested form (2D n = 5..8)."""
    for n in range(5, 9):
        sets = [COMPARISON_SETS[(2, n)] + [INF], PROPOSED_SETS[(2, n)] + [INF]]
        nested = wino.wino_pointset_error((2, n - 2, 3), sets, 1000)
        kron = wino.wino_pointset_error_kron(n - 2, sets, 1000)
        pw = wino.wino_pointset_error_kron(n - 2, sets, 1000, pairwise=True)
        assert np.all(kron > nested) and np.all(pw > nested), (n, nested, kron, pw)
