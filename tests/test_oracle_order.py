"""Oracle pins for the summation-order variants of the single tile (Sec. 5:
the Huffman evaluation order the paper's tables use, alone and with FP64
transforms).  The tree is pinned against brute-force optimality and its tie
rule, the FP32 sum against worked values, the tile against exact arithmetic
(rational transforms rounded where the reading rounds) -- none of them
re-types the oracle's loops."""
import itertools
import math
from fractions import Fraction
from functools import lru_cache

import numpy as np
import pytest

from paper_2201_10369_gb300.inputs import COMPARISON_SETS, PROPOSED_SETS

INF = math.inf


# --- the tree -----------------------------------------------------------------

@lru_cache(maxsize=None)
def _best_cost(ws):
    """Least weighted path length over every binary tree on the leaves ws
    (the sum of the merged weights over any merge sequence), brute force."""
    if len(ws) <= 1:
        return 0
    best = None
    for i, j in itertools.combinations(range(len(ws)), 2):
        rest = [w for k, w in enumerate(ws) if k not in (i, j)] + [ws[i] + ws[j]]
        c = ws[i] + ws[j] + _best_cost(tuple(sorted(rest)))
        best = c if best is None or c < best else best
    return best


def _tree_cost(w, merges):
    wt = list(w)
    cost = 0
    for f, s in merges:
        wt.append(wt[f] + wt[s])
        cost += wt[-1]
    return cost


def test_huffman_tree_is_optimal(orc):
    """A Huffman tree has the least weighted path length: compare with brute
    force over all trees (integer weights, exact sums); zero weights are left
    out of the tree."""
    rng = np.random.default_rng(5)
    for n in range(1, 8):
        for _ in range(12):
            w = rng.integers(0, 12, n).astype(float)
            if not np.any(w > 0):
                w[0] = 1.0
            merges = orc.huffman_merges(w)
            live = [x for x in w if x > 0]
            assert len(merges) == len(live) - 1
            used = {i for m in merges for i in m}
            assert all(w[k] > 0 for k in range(n) if k in used)
            assert len(set(i for m in merges for i in m)) == 2 * len(merges)  # each node once
            assert _tree_cost(w, merges) == _best_cost(tuple(sorted(live))), (w, merges)


def test_huffman_tie_rule(orc):
    """Ties go to the node created first: leaves in column order, then merged
    nodes in creation order."""
    assert orc.huffman_merges([1, 1, 1, 1]) == [(0, 1), (2, 3), (4, 5)]
    assert orc.huffman_merges([2, 1, 1]) == [(1, 2), (0, 3)]
    assert orc.huffman_merges([3, 0, 1]) == [(2, 0)]
    assert orc.huffman_merges([1, 1, 1]) == [(0, 1), (2, 3)]
    assert orc.huffman_merges([0, 5]) == []


def test_huffman_dot_worked_example(orc):
    """c = (1,1,1,1), x = (1, 0, 2^-24, 2^-24): the balanced tree adds the two
    small terms first, 1 + 2^-23 exactly; the column-order FP32 sum (and the
    fmaf order) lands on 1."""
    c = np.ones(4, np.float32)
    x = np.array([1.0, 0.0, 2.0 ** -24, 2.0 ** -24], np.float32)
    assert orc.huffman_dot_f32(c, x) == np.float32(1 + 2.0 ** -23)
    seq = np.float32(0)
    for k in range(4):
        seq = np.float32(seq + np.float32(c[k] * x[k]))
    assert seq == np.float32(1.0)


def test_huffman_dot_dominant_weights(orc):
    """When every |c_k| exceeds the sum of the smaller ones the tree is a
    chain: the sum is the sequential FP32 sum in ascending |c| order."""
    rng = np.random.default_rng(11)
    for n in range(2, 11):
        for _ in range(20):
            mag = 3.0 ** np.arange(n) * rng.uniform(1.0, 1.4, n)
            perm = rng.permutation(n)
            c = (mag[perm] * rng.choice([-1, 1], n)).astype(np.float32)
            x = rng.uniform(-1, 1, n).astype(np.float32)
            acc = np.float32(0)
            for k in np.argsort(np.abs(c.astype(np.float64)), kind="stable"):
                acc = np.float32(acc + np.float32(c[k] * x[k]))
            assert orc.huffman_dot_f32(c, x) == acc


def test_huffman_dot_skips_zero_terms(orc):
    c = np.array([0.0, 2.0, 0.0, 3.0], np.float32)
    x = np.array([np.inf, 0.5, np.nan, 0.25], np.float32)  # never read
    assert orc.huffman_dot_f32(c, x) == np.float32(1.75)


# --- the tile -----------------------------------------------------------------

def _exact_corr(dim, g, d, m, r):
    if dim == 1:
        return np.array([sum(Fraction(float(g[k])) * Fraction(float(d[j + k])) for k in range(r))
                         for j in range(m)], dtype=object)
    return np.array([[sum(Fraction(float(g[u, v])) * Fraction(float(d[a + u, b + v]))
                          for u in range(r) for v in range(r)) for b in range(m)]
                     for a in range(m)], dtype=object)


@pytest.mark.parametrize("order", ["huffman", "huffman_mixed"])
@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("pts", [[0.0, 1.0, -1.0, INF], [0.0, 1.0, 2.0, INF]])
def test_tile_exact_regime(orc, order, dim, pts):
    """Integer inputs with dyadic matrices: no operation rounds, so every
    order returns the exact correlation."""
    rng = np.random.default_rng(3)
    m, r = 2, 3
    for _ in range(20):
        g = rng.integers(-3, 4, (r,) * dim).astype(np.float32)
        d = rng.integers(-3, 4, (4,) * dim).astype(np.float32)
        y = orc.tile_order(dim, pts, m, r, g, d, order)
        assert np.array_equal(y.astype(object), _exact_corr(dim, g, d, m, r))


def _rn32(q: Fraction, ties: list) -> np.float32:
    """Round a rational to the nearest FP32 value, ties to even.  Appends to
    `ties` when q lies within 2^-40 relative of a midpoint but not on it:
    there the FP64 sums' own rounding (~1e-16) may decide the FP32 rounding
    either way (FP32 inputs times the FP64 value of a third land next to
    midpoints often).  A value exactly on a midpoint is a sum the FP64 pass
    computes exactly, and both sides round it to even."""
    f = np.float32(float(q))
    cands = [f, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))]
    dist = sorted((abs(Fraction(float(c)) - q), int(np.array(c, np.float32).view(np.uint32)) & 1,
                   float(c)) for c in cands)
    if 0 < dist[1][0] - dist[0][0] <= abs(q) / 2 ** 40:
        ties.append(q)
    return np.float32(dist[0][2])


def _mixed_reference(orc, dim, pts, m, r, g, d):
    """Transforms exact on the FP64 matrix entries, rounded to FP32 at U and
    V; P = U .* V in FP32; output transform exact, rounded once.  Returns the
    tile and whether a rounding point sat on a near-tie."""
    AT, G, BT = orc.make_matrices(pts, m, r)
    A = m + r - 1
    Q = np.vectorize(lambda v: Fraction(float(v)), otypes=[object])
    AT, G, BT = Q(AT), Q(G), Q(BT)
    ties = []
    rn = np.vectorize(lambda q: _rn32(q, ties), otypes=[np.float32])
    if dim == 1:
        U = rn(G.dot(Q(g)))
        V = rn(BT.dot(Q(d)))
        P = (U * V).astype(np.float32)
        return rn(AT.dot(Q(P))), bool(ties)
    U = rn(G.dot(Q(g)).dot(G.T))
    V = rn(BT.dot(Q(d)).dot(BT.T))
    P = (U * V).astype(np.float32)
    assert P.shape == (A, A)
    return rn(AT.dot(Q(P)).dot(AT.T)), bool(ties)


def _cases():
    out = []
    for (dim, n), pts in sorted(PROPOSED_SETS.items()):
        if dim == 2 and n > 8:
            continue
        out.append((dim, n - 2, list(pts) + [INF]))
    for (dim, n), pts in sorted(COMPARISON_SETS.items()):
        if dim == 2 and n > 8:
            continue
        out.append((dim, n - 2, list(pts) + [INF]))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: "d%d_m%d_%s" % (c[0], c[1], c[2][1]))
def test_mixed_tile_equals_rational_transforms(orc, case):
    """The FP64-transform variant rounds only at U, V, P and Y: equal to the
    rational transforms of the FP64 matrices rounded there, on every trial
    whose rounding points keep clear of FP32 midpoints (the FP64 sums' own
    errors decide a near-tie); those trials are at most half."""
    dim, m, pts = case
    r, A = 3, m + 2
    rng = np.random.default_rng(17 + m + 10 * dim)
    n, clear = 8, 0
    for _ in range(n):
        g = rng.uniform(-1, 1, (r,) * dim).astype(np.float32)
        d = rng.uniform(-1, 1, (A,) * dim).astype(np.float32)
        y = orc.tile_order(dim, pts, m, r, g, d, "huffman_mixed")
        ref, tie = _mixed_reference(orc, dim, pts, m, r, g, d)
        if tie:
            assert np.max(np.abs(y - ref) / np.max(np.abs(ref))) < 1e-5
        else:
            clear += 1
            assert np.array_equal(y, ref)
    print("clear trials", clear, "of", n)
    assert clear >= n // 2


@pytest.mark.parametrize("case", _cases(), ids=lambda c: "d%d_m%d_%s" % (c[0], c[1], c[2][1]))
def test_huffman_tile_within_fp32_error(orc, case):
    """The FP32 Huffman tile is the exact correlation up to FP32 rounding of
    the transforms (the scale the plain order shows), and not the plain
    order's bits on every trial."""
    dim, m, pts = case
    r, A = 3, m + 2
    AT, G, BT = orc.make_matrices(pts, m, r)
    rng = np.random.default_rng(29 + m + 10 * dim)
    differs = 0
    for _ in range(6):
        g = rng.uniform(-1, 1, (r,) * dim).astype(np.float32)
        d = rng.uniform(-1, 1, (A,) * dim).astype(np.float32)
        y = orc.tile_order(dim, pts, m, r, g, d, "huffman")
        yp = orc.tile_f32(dim, AT.astype(np.float32), G.astype(np.float32),
                          BT.astype(np.float32), m, r, g, d)
        ex = _exact_corr(dim, g, d, m, r).astype(np.float64)
        scale = np.max(np.abs(yp - ex)) + 1e-7 * np.max(np.abs(ex))
        assert np.max(np.abs(y - ex)) <= 20 * scale
        differs += int(not np.array_equal(y, yp))
    if m >= 3:
        assert differs > 0


def test_order_errors_near_plain(orc):
    """Sweep metric in each order, same trials: the three stay within a factor
    1.5 of one another for the paper's sets (the order moves the error by
    percents, Sec. 5), and the FP64 transforms lower it."""
    for (dim, n), pts in [((1, 6), PROPOSED_SETS[(1, 6)]), ((2, 6), PROPOSED_SETS[(2, 6)]),
                          ((2, 8), COMPARISON_SETS[(2, 8)])]:
        s = [list(pts) + [INF]]
        e = {o: orc.pointset_error_order(dim, n - 2, 3, s, 300, 0, o)[0]
             for o in ("fma", "huffman", "huffman_mixed")}
        assert e["fma"] == orc.pointset_error(dim, n - 2, 3, s, 300, 0)[0]
        assert 1 / 1.5 < e["huffman"] / e["fma"] < 1.5, e
        assert e["huffman_mixed"] < e["huffman"], e


from test_oracle_pointsets import _rows  # noqa: E402
from test_oracle_sweep import _mean_abs_y  # noqa: E402


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r["label"])
def test_huffman_order_matches_printed_errors(orc, row):
    """Tables 7-8 were measured in Huffman order (Sec. 5): the comparison sets
    in this reading of it, per-element absolute error, land within
    [0.9, 1.05] of the printed values for n >= 5 and [0.8, 1.05] for n = 4
    (the plain fmaf order reaches only [0.9, 1.0] at n >= 5; 5000 trials
    like the paper's, but not its inputs)."""
    trials, seed = 5000, 0
    rel = orc.pointset_error_order(row["dim"], row["m"], 3, [row["points"]], trials, seed,
                                   "huffman")[0]
    ratio = rel * _mean_abs_y(orc, row["dim"], row["m"], trials, seed) / row["paper"]
    lo = 0.8 if row["m"] == 2 else 0.9
    assert lo <= ratio <= 1.05, (row["cite"], ratio)
