"""Oracle pins for explicit point sets: the comparison sets of Barabasz et al.
against the errors Tables 7-8 print for them, the Chebyshev nodes of Sec. 2
against their closed form, and the point-set metric against the mask sweep
where a set has both forms."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from test_oracle_sweep import _mean_abs_y

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_pointsets.txt")


def _rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = [s.strip() for s in line.split("|")]
            pts = [float(Fraction(v)) for v in p[3].split(",")] + [math.inf]
            rows.append(dict(label=p[0], dim=int(p[1]), m=int(p[2]), points=pts,
                             paper=float(p[4]), cite=p[5]))
    return rows


from paper_2201_10369_gb300.inputs import (COMPARISON_SETS, PAPER_IMPROVEMENT_PCT,  # noqa: E402
                                           PROPOSED_SETS, chebyshev_points)

# Rows of Tables 7-8 whose printed improvement our plain-order FP32 does not
# reproduce: 1D n=10 and 2D n=5 print proposed-set errors 2.5x and 1.5x below
# what we measure for those sets (paper_errors.txt, "loose"); 1D n=5 measures
# -2% against the printed +9.6%.
SIGN_EXCEPTIONS = {(1, 5), (1, 10), (2, 5)}


def test_input_sets_match_golden():
    """The comparison sets the bench and GPU tests use are the golden file's."""
    for r in _rows():
        assert COMPARISON_SETS[(r["dim"], r["m"] + 2)] + [math.inf] == r["points"], r["label"]


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r["label"])
def test_barabasz_sets_match_printed_errors(orc, row):
    """Our error for the paper's comparison sets, in the per-element absolute
    reading, within [0.75, 1.05] of the printed value (Huffman order there)."""
    trials, seed = 5000, 0
    rel = orc.pointset_error(row["dim"], row["m"], 3, [row["points"]], trials, seed)[0]
    ours = rel * _mean_abs_y(orc, row["dim"], row["m"], trials, seed)
    assert 0.75 <= ours / row["paper"] <= 1.05, (row["cite"], ours, row["paper"])


def test_chebyshev_closed_form():
    assert np.allclose(chebyshev_points(1), [0.0], atol=1e-15)
    assert np.allclose(chebyshev_points(3), [math.sqrt(3) / 2, 0.0, -math.sqrt(3) / 2], atol=1e-15)
    p = chebyshev_points(7)
    assert np.allclose(p, -np.array(p[::-1]), atol=1e-15)  # symmetric about 0
    assert all(-1 < v < 1 for v in p)


def test_chebyshev_worse_for_larger_sets(orc):
    """Table 9: for n >= 6 points the Chebyshev nodes give a larger error than
    the Barabasz sets (every column); the synthetic sweep agrees in 1D and 2D."""
    rows = {(r["dim"], r["m"]): r for r in _rows()}
    for dim in (1, 2):
        for m in (4, 6, 8):
            ch = chebyshev_points(m + 1) + [math.inf]
            e = orc.pointset_error(dim, m, 3, [rows[(dim, m)]["points"], ch], 1000, 0)
            assert e[1] > e[0], (dim, m, e)


def test_pointset_equals_mask_sweep(orc):
    """P8 is the full c-group with c = 2, d = 1 (mask 0x6f): the point-set
    metric and the mask sweep evaluate the same matrices on the same trials."""
    p8 = [0, -1, 1, 0.5, -0.5, 2, -2, math.inf]
    for dim in (1, 2):
        a = orc.pointset_error(dim, 6, 3, [p8], 300, 4)[0]
        b = orc.error_sweep([2.0], [(dim, 6, 3, 1.0)], [0x6F], 300, 4)[0, 0, 0]
        assert a == b


def test_pointset_degenerate(orc):
    e = orc.pointset_error(1, 2, 3, [[0, 1, 1, math.inf], [0, 1, -1, 2.0]], 50, 0)
    assert math.isinf(e[0]) and math.isnan(e[1])


@pytest.mark.slow
def test_paper_comparison_signs(orc):
    """Tables 7-8: the paper's proposed set of each size against Barabasz's
    set of that size.  Where the paper reports a change of more than 5%, our
    error reproduces its sign (8 such rows; SIGN_EXCEPTIONS lists the three
    it does not), e.g. 2D F(4x4) c = 1.622: about +30% (paper +28%)."""
    checked = 0
    for (dim, n), paper in PAPER_IMPROVEMENT_PCT.items():
        if abs(paper) <= 5.0 or (dim, n) in SIGN_EXCEPTIONS:
            continue
        e = orc.pointset_error(dim, n - 2, 3, [COMPARISON_SETS[(dim, n)] + [math.inf],
                                                 PROPOSED_SETS[(dim, n)] + [math.inf]], 2000, 0)
        ours = 100.0 * (e[0] - e[1]) / e[0]
        assert np.sign(ours) == np.sign(paper), (dim, n, ours, paper)
        checked += 1
    assert checked == 8


@pytest.mark.parametrize("pairwise", [False, True])
def test_kron_tile_exact_on_integers(orc, pairwise):
    """Exact regime of the Kronecker-product form (Sec. 7): P4's matrices and
    their Kronecker products are exact in FP32, so on small integer inputs
    the tile equals the direct correlation -- a transposed Kronecker matrix or
    a swapped factor order (d read as d^T) fails here."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        g = rng.integers(-9, 10, (3, 3)).astype(np.float32)
        d = rng.integers(-9, 10, (4, 4)).astype(np.float32)
        y = orc.tile2d_kron([0.0, -1.0, 1.0, math.inf], 2, 3, g, d, pairwise)
        want = np.array([[np.sum(d[a:a + 3, b:b + 3] * g) for b in range(2)] for a in range(2)])
        assert np.array_equal(y, want.astype(np.float32))


def test_kron_and_nested_agree_to_first_order(orc):
    """Off the exact regime the two forms differ only by rounding: on the
    sweep's trials their errors agree to first order (within 2x)."""
    sets = [COMPARISON_SETS[(2, 6)] + [math.inf]]
    a = orc.pointset_error(2, 4, 3, sets, 300, 0)[0]
    b = orc.pointset_error_kron(4, 3, sets, 300, 0)[0]
    assert 0.5 < b / a < 2.0


def test_kron_error_larger_than_nested(orc):
    """Sec. 7: the Kronecker-product transforms give a larger FP error than the
    nested matrix products, and pairwise summation does not remove the gap
    (2D, n = 5..8, Barabasz's and the proposed sets)."""
    for n in range(5, 9):
        sets = [COMPARISON_SETS[(2, n)] + [math.inf], PROPOSED_SETS[(2, n)] + [math.inf]]
        nested = orc.pointset_error(2, n - 2, 3, sets, 1000, 0)
        kron = orc.pointset_error_kron(n - 2, 3, sets, 1000, 0)
        pw = orc.pointset_error_kron(n - 2, 3, sets, 1000, 0, pairwise=True)
        assert np.all(kron > nested) and np.all(pw > nested), (n, nested, kron, pw)
