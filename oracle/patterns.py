"""Subset-pattern query of the point sweep -- TEST INFRASTRUCTURE ONLY.

Sec. 6.2 combines fixed "base points" (besides 0 and infinity, e.g. 3, -3,
1/2 or the pair 1, -1) with a subset of the group {-1/c, -c, c, 1/c}; its
Tables 2-4 give, per base and subset, the c of least error and that error,
and Tables 5-6 name the subset that gives the least error for each base
(the "optimal pattern").  Here the base points are the sweep's d-group slots
(bits 4-7 of a mask over [-1/c, -c, c, 1/c, -1/d, -d, d, 1/d]) and the
subset its c-group bits (0-3); the errors come from one size's sweep,
err[mask][c].  Plain loops over the candidates and the grid; the GPU
library's host query must return the same answer on the same array.

Reading (the paper gives no procedure): the candidates of a base are the
masks whose d-group bits equal the base's and that are valid for the size
(popcount alpha - 2; bits 4 and 7 unused when |d| = 1).  Only the c in
[c_lo, c_hi] count.  A candidate's best is the least finite error there
(the first grid index on ties).  Its win fraction is the share of the
window's c, among those where every candidate is finite, at which it has
the least error (ties to the smaller mask).  Candidates are listed by best
error, then mask; those with no finite error come last.
"""
from __future__ import annotations

import math


def valid_for(mask: int, alpha: int, d: float) -> bool:
    if bin(mask).count("1") != alpha - 2:
        return False
    if abs(d) == 1.0 and (mask & 0x90):
        return False
    return True


def subset_pattern(err, masks, c_grid, alpha: int, d: float, base_mask: int,
                   c_lo: float, c_hi: float):
    """Candidates of `base_mask` ranked as above: a list of dicts
    {mask, best_k, best_c, best_err, win_frac}."""
    masks = [int(v) for v in masks]
    cands = [q for q, mk in enumerate(masks)
             if (mk & 0xF0) == base_mask and valid_for(mk, alpha, d)]
    window = [k for k in range(len(c_grid)) if c_lo <= c_grid[k] <= c_hi]
    rows = []
    for q in cands:
        best_k, best_e = -1, math.nan
        for k in window:
            e = float(err[q][k])
            if math.isfinite(e) and (best_k < 0 or e < best_e):
                best_k, best_e = k, e
        rows.append({"q": q, "mask": masks[q], "best_k": best_k,
                     "best_c": float(c_grid[best_k]) if best_k >= 0 else math.nan,
                     "best_err": best_e, "wins": 0})
    common = 0
    for k in window:
        vals = [float(err[r["q"]][k]) for r in rows]
        if not rows or not all(math.isfinite(v) for v in vals):
            continue
        common += 1
        w = 0
        for i in range(1, len(rows)):
            if vals[i] < vals[w] or (vals[i] == vals[w] and rows[i]["mask"] < rows[w]["mask"]):
                w = i
        rows[w]["wins"] += 1
    for r in rows:
        r["win_frac"] = r["wins"] / common if common else 0.0
        del r["wins"], r["q"]
    rows.sort(key=lambda r: (0 if r["best_k"] >= 0 else 1,
                             r["best_err"] if r["best_k"] >= 0 else 0.0, r["mask"]))
    return rows
