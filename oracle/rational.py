"""Exact (rational) Toom-Cook construction and convolution -- TEST INFRASTRUCTURE.

Written with ``fractions.Fraction`` so that every identity the paper states
holds exactly: the modified Toom-Cook matrices of Sec. 4.1-4.2 (Eqs. (10),
(11), (19)), the 1D/2D Winograd evaluation of Eqs. (8)-(9), and the direct
correlation of Eq. (1).  Used only by tests to pin the floating-point oracle.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Sequence

INF = "inf"


def canonical(points: Sequence) -> List:
    """Finite points ascending, the point at infinity last."""
    fin = sorted(Fraction(p) for p in points if p != INF)
    n_inf = sum(1 for p in points if p == INF)
    if n_inf != 1:
        raise ValueError("exactly one point at infinity is required")
    return fin + [INF]


def poly_from_roots(roots: Sequence[Fraction]) -> List[Fraction]:
    """Ascending coefficients of prod (x - a) over `roots`."""
    p = [Fraction(1)]
    for a in roots:
        q = [Fraction(0)] * (len(p) + 1)
        for l, cl in enumerate(p):
            q[l + 1] += cl
            q[l] -= a * cl
        p = q
    return p


def matrices(points: Sequence, m: int, r: int):
    """(AT, G, BT) as lists of lists of Fractions, canonical point order."""
    pts = canonical(points)
    alpha = m + r - 1
    if len(pts) != alpha:
        raise ValueError("need alpha = m + r - 1 points")
    fin = pts[:-1]
    nf = len(fin)
    if len(set(fin)) != nf:
        raise ZeroDivisionError("coinciding points")
    N = []
    for i, ai in enumerate(fin):
        prod = Fraction(1)
        for j, aj in enumerate(fin):
            if j != i:
                prod *= ai - aj
        N.append(prod)
    G = [[fin[i] ** k / N[i] for k in range(r)] for i in range(nf)]
    G.append([Fraction(1 if k == r - 1 else 0) for k in range(r)])
    AT = [[fin[i] ** j for i in range(nf)] + [Fraction(1 if j == m - 1 else 0)] for j in range(m)]
    BT = []
    for i in range(nf):
        coeffs = poly_from_roots([fin[j] for j in range(nf) if j != i])
        BT.append(coeffs + [Fraction(0)] * (alpha - len(coeffs)))
    BT.append(poly_from_roots(fin))
    return AT, G, BT


def matvec(Mx, v):
    return [sum((a * b for a, b in zip(row, v)), Fraction(0)) for row in Mx]


def transpose(Mx):
    return [list(col) for col in zip(*Mx)]


def matmul(X, Y):
    Yt = transpose(Y)
    return [[sum((a * b for a, b in zip(row, col)), Fraction(0)) for col in Yt] for row in X]


def wino_tile_1d(AT, G, BT, g, d):
    u = matvec(G, g)
    v = matvec(BT, d)
    return matvec(AT, [a * b for a, b in zip(u, v)])


def wino_tile_2d(AT, G, BT, g, d):
    U = matmul(matmul(G, g), transpose(G))
    V = matmul(matmul(BT, d), transpose(BT))
    P = [[a * b for a, b in zip(ru, rv)] for ru, rv in zip(U, V)]
    return matmul(matmul(AT, P), transpose(AT))


def correlate_1d(g, d):
    m = len(d) - len(g) + 1
    return [sum((g[k] * d[j + k] for k in range(len(g))), Fraction(0)) for j in range(m)]


def correlate_2d(g, d):
    r = len(g)
    m = len(d) - r + 1
    return [[sum((g[u][v] * d[a + u][b + v] for u in range(r) for v in range(r)), Fraction(0))
             for b in range(m)] for a in range(m)]


def direct_layer_2d(x, w, pad: int):
    """Exact Eq. (1) with zero padding: x[N][C][H][W], w[K][C][r][r]."""
    N, C, H, W = len(x), len(x[0]), len(x[0][0]), len(x[0][0][0])
    K, r = len(w), len(w[0][0])
    Ho, Wo = H + 2 * pad - r + 1, W + 2 * pad - r + 1
    y = [[[[Fraction(0)] * Wo for _ in range(Ho)] for _ in range(K)] for _ in range(N)]
    for n in range(N):
        for k in range(K):
            for p in range(Ho):
                for q in range(Wo):
                    acc = Fraction(0)
                    for c in range(C):
                        for u in range(r):
                            for v in range(r):
                                hh, ww = p + u - pad, q + v - pad
                                if 0 <= hh < H and 0 <= ww < W:
                                    acc += Fraction(x[n][c][hh][ww]) * Fraction(w[k][c][u][v])
                    y[n][k][p][q] = acc
    return y
