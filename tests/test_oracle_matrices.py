"""Pins of the oracle's transform-matrix construction (Sec. 4.1-4.2, Sec. 5).

Independent checks: the paper's printed symbolic matrices (Eqs. (26)-(31)),
the exactness identity of Toom-Cook in rational arithmetic, Lavin and Gray's
published F(2,3) matrices up to per-point rescaling, and agreement of the
FP64 build with the exact build.
"""
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import rational as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_matrices.txt")


def _parse_golden():
    blocks, cur = [], None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("@"):
                _, name, m, r, *cite = line.split()
                cur = {"name": name, "m": int(m), "r": int(r), "cite": " ".join(cite),
                       "vars": {}, "rows": []}
                blocks.append(cur)
            elif line.startswith("vars"):
                for kv in line.split()[1:]:
                    k, v = kv.split("=")
                    cur["vars"][k] = Fraction(v)
            else:
                head, entries = line.split(":")
                mat, pt = head.split()
                cur["rows"].append((mat, pt, [e.strip() for e in entries.split(",")]))
    return blocks


def _ev(expr, env):
    if expr == "inf":
        return "inf"
    return Fraction(eval(expr, {"__builtins__": {}}, dict(env)))


@pytest.mark.parametrize("block", _parse_golden(), ids=lambda b: b["name"])
def test_paper_symbolic_matrices(block):
    env = block["vars"]
    pts = []
    for mat, pt, _ in block["rows"]:
        if mat == "BT":
            pts.append(_ev(pt, env))
    AT, G, BT = R.matrices(pts, block["m"], block["r"])
    order = R.canonical(pts)
    for mat, pt, entries in block["rows"]:
        p = _ev(pt, env)
        i = order.index(p)
        got = (BT if mat == "BT" else G)[i]
        want = [_ev(e, env) for e in entries]
        assert got == want, (block["cite"], mat, pt, got, want)


def _rand_points(rng, nf):
    pts = set()
    while len(pts) < nf:
        pts.add(Fraction(rng.randint(-40, 40), rng.randint(1, 9)))
    return sorted(pts) + ["inf"]


@pytest.mark.parametrize("r", [3, 5])
@pytest.mark.parametrize("m", range(1, 9))
def test_exactness_tensor_rational(m, r):
    """sum_i AT[j,i] G[i,k] BT[i,l] = delta(l, j+k): Y = AT[(Gg).(BTd)] is
    exactly the correlation Y_j = sum_k g_k d_{j+k} (Eqs. (8), (13)-(19))."""
    alpha = m + r - 1
    if alpha > 10:
        pytest.skip("alpha > 10 not used")
    rng = random.Random(100 * m + r)
    AT, G, BT = R.matrices(_rand_points(rng, alpha - 1), m, r)
    for j in range(m):
        for k in range(r):
            for l in range(alpha):
                s = sum((AT[j][i] * G[i][k] * BT[i][l] for i in range(alpha)), Fraction(0))
                assert s == (1 if l == j + k else 0), (j, k, l, s)


def test_lavin_f23_rank1_terms():
    """Lavin and Gray's F(2,3) (points 0, 1, -1, inf) equals ours up to the
    per-point scaling freedom: the rank-one terms AT[:,i] x G[i,:] x BT[i,:]
    are invariant."""
    BTl = [[1, 0, -1, 0], [0, 1, 1, 0], [0, -1, 1, 0], [0, 1, 0, -1]]
    Gl = [[1, 0, 0], [Fraction(1, 2)] * 3, [Fraction(1, 2), Fraction(-1, 2), Fraction(1, 2)],
          [0, 0, 1]]
    ATl = [[1, 1, 1, 0], [0, 1, -1, -1]]
    lavin_points = [0, 1, -1, "inf"]
    AT, G, BT = R.matrices(lavin_points, 2, 3)
    order = R.canonical(lavin_points)

    def term(ATm, Gm, BTm, i):
        return [[[Fraction(ATm[j][i]) * Gm[i][k] * BTm[i][l] for l in range(4)] for k in range(3)]
                for j in range(2)]

    for il, p in enumerate(lavin_points):
        assert term(ATl, Gl, BTl, il) == term(AT, G, BT, order.index(p if p == "inf" else Fraction(p)))


@pytest.mark.parametrize("m", range(2, 9))
def test_fp64_build_matches_exact(orc, m):
    """FP64 build vs the exact build rounded to FP64: 1e-13 relative (the
    GPU-versus-oracle bar for the matrices)."""
    r = 3
    rng = random.Random(7 + m)
    pts = _rand_points(rng, m + 1)
    ATq, Gq, BTq = R.matrices(pts, m, r)
    fpts = [math.inf if p == "inf" else float(p) for p in pts]
    AT, G, BT = orc.make_matrices(fpts, m, r)
    for got, want in ((AT, ATq), (G, Gq), (BT, BTq)):
        w = np.array([[float(v) for v in row] for row in want])
        scale = np.abs(w).max()
        assert np.abs(got - w).max() <= 1e-13 * scale


@pytest.mark.parametrize("m", [2, 4, 6])
def test_fp64_build_proposed_points(orc, m):
    """The symmetric families of Sec. 5 in FP64: exactness identity holds to
    rounding and the ones/zeros the construction forces are exact."""
    c = 1.7
    base = [-1 / c, -c, c, 1 / c, -1.0, 1.0][: m]
    pts = [0.0] + base + [math.inf]
    AT, G, BT = orc.make_matrices(pts, m, 3)
    a = m + 2
    T = np.einsum("ji,ik,il->jkl", AT, G, BT)
    E = np.zeros_like(T)
    for j in range(m):
        for k in range(3):
            E[j, k, j + k] = 1.0
    assert np.abs(T - E).max() < 1e-12
    assert np.all(BT[:-1, a - 2] == 1.0) and np.all(BT[:-1, a - 1] == 0.0) and BT[-1, -1] == 1.0
    assert np.all(G[-1] == [0, 0, 1]) and np.all(AT[:, -1] == np.eye(m)[-1])


def test_canonical_order_and_errors(orc):
    AT1, G1, BT1 = orc.make_matrices([np.inf, 1.0, 0.0, -1.0], 2, 3)
    AT2, G2, BT2 = orc.make_matrices([-1.0, 0.0, 1.0, np.inf], 2, 3)
    assert np.array_equal(AT1, AT2) and np.array_equal(G1, G2) and np.array_equal(BT1, BT2)
    with pytest.raises(orc.SingularPoints):
        orc.make_matrices([0.0, 1.0, 1.0, np.inf], 2, 3)
    for bad in ([0.0, 1.0, -1.0, 2.0], [0.0, np.inf, -1.0, np.inf], [0.0, np.nan, 1.0, np.inf],
                [0.0, -np.inf, 1.0, 2.0]):
        with pytest.raises(ValueError):
            orc.make_matrices(bad, 2, 3)
