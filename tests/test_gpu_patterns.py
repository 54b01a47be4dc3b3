"""Subset patterns (Sec. 6.2, Tables 5-6) from the GPU sweep: the library's
query (wino_subset_pattern) on the GPU sweep against the oracle's query on
the oracle's sweep of the same grid, and the patterns of the full c grid
against the ones the paper prints (a loose pin: the paper sums in Huffman
order with 5000 trials, the sweep in fmaf order with 1000)."""
import os

import numpy as np
import pytest

from oracle import patterns as opat
from paper_2201_10369_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_patterns.txt")


def golden_patterns():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = [s.strip() for s in line.split("|")]
            rows.append(dict(label=p[0], dim=int(p[1]), m=int(p[2]), d=float(p[3]),
                             base=int(p[4], 16), pattern=None if p[5] == "none" else int(p[5], 16),
                             cite=p[6]))
    return rows


def mirror(sub):
    """The subset at c that is `sub` at 1/c: -1/c <-> -c, c <-> 1/c."""
    return ((sub & 1) << 1) | ((sub & 2) >> 1) | ((sub & 4) << 1) | ((sub & 8) >> 1)


def candidate_masks(m, bases):
    """Masks base | S, S a subset of the c-group, with alpha - 2 = m points."""
    out = set()
    for b in bases:
        for s in range(16):
            if bin(b | s).count("1") == m:
                out.add(b | s)
    return np.array(sorted(out), dtype=np.uint8)


def _groups():
    g = {}
    for r in golden_patterns():
        g.setdefault((r["dim"], r["m"], r["d"]), []).append(r)
    return g


def test_query_on_gpu_sweep_matches_oracle(wino, orc):
    cg = inputs.c_grid()[2048::48]  # c > 1, 43 grid points
    for (dim, m, d), rows in _groups().items():
        masks = candidate_masks(m, [r["base"] for r in rows])
        size = (dim, m, 3, d)
        eg = wino.wino_error_sweep(cg, [size], masks, 300, seed=0)[0]
        eo = orc.error_sweep(cg, [size], masks, 300, 0)[0]
        for r in rows:
            got = {c["mask"]: c for c in wino.wino_subset_pattern(eg, masks, cg, size, r["base"],
                                                                   1.0, 20.0)}
            want = {c["mask"]: c for c in opat.subset_pattern(eo, masks, cg, m + 2, d, r["base"],
                                                              1.0, 20.0)}
            assert set(got) == set(want)
            for mk, w in want.items():
                g = got[mk]
                assert abs(g["best_err"] - w["best_err"]) <= 1e-6 * w["best_err"], r["label"]
                if g["best_k"] != w["best_k"]:  # a near-tie inside the row
                    assert abs(eo[list(masks).index(mk), g["best_k"]] - w["best_err"]) <= \
                        2e-6 * w["best_err"]
                assert abs(g["win_frac"] - w["win_frac"]) <= 2.0 / cg.size, r["label"]


def measured_patterns(wino, trials=1000):
    """Our pattern per golden entry on the full grid's c > 1."""
    cg = inputs.c_grid()
    out = {}
    for (dim, m, d), rows in _groups().items():
        masks = candidate_masks(m, [r["base"] for r in rows])
        size = (dim, m, 3, d)
        err = wino.wino_error_sweep(cg, [size], masks, trials, seed=0)[0]
        for r in rows:
            out[r["label"]] = wino.wino_subset_pattern(err, masks, cg, size, r["base"], 1.0, 20.0)
    return out


def reproduces(r, cands):
    """A printed pattern reproduces when the measured best subset is it or
    its mirror; "no pattern" when the measured best wins at most half of the
    window's c."""
    top = cands[0]
    if r["pattern"] is None:
        return top["win_frac"] <= 0.5
    sub = top["mask"] & 0x0F
    return sub in (r["pattern"], mirror(r["pattern"]))


def test_patterns_vs_paper(wino):
    """14 of the 16 printed entries reproduce (both "No pattern" entries
    among them: the best subset wins about 0.37 of the c > 1 window).  The
    base 1/2 F(3,3) entries, {-c, c} in both tables, measure {-1/c, c} by a
    near-tie (its win fraction 0.46 in 1D, 0.20 in 2D); the bar leaves
    room for one more near-tie to flip."""
    rows = golden_patterns()
    meas = measured_patterns(wino)
    ok = [reproduces(r, meas[r["label"]]) for r in rows]
    print({r["label"]: ("%#04x" % (meas[r["label"]][0]["mask"] & 15),
                        round(meas[r["label"]][0]["win_frac"], 2), o) for r, o in zip(rows, ok)})
    assert sum(ok) >= 13, [r["label"] for r, o in zip(rows, ok) if not o]
