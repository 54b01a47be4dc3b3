"""The subset-pattern query of Sec. 6.2 (Tables 2-6), CPU only: the oracle's
plain statement pinned to hand-built error curves whose answer is known, and
the library's host query (wino_subset_pattern) equal to it on random error
arrays (ties, NaN, +inf, windows) and on an oracle sweep."""
import math

import numpy as np
import pytest

from oracle import patterns as opat

SIZE_D3 = (1, 3, 3, 3.0)   # F(3,3), alpha = 5: base point 3 (bit 6) + 2 of the c-group
SIZE_D1 = (1, 4, 3, 1.0)   # F(4,3), alpha = 6: base {-1, 1} (bits 5, 6) + 2 of the c-group


def _curves(masks, cg, f):
    return np.array([[f(mk, c) for c in cg] for mk in masks])


def test_oracle_pattern_known_answers():
    cg = np.geomspace(0.5, 8.0, 65)
    masks = [0x43, 0x45, 0x49, 0x46, 0x4A, 0x4C, 0x21, 0x03]
    lo = {0x45: 0.0, 0x43: 0.1, 0x49: 0.2}

    def f(mk, c):
        base = (math.log(c) - math.log(1.5)) ** 2
        return 1.0 + base + lo.get(mk, 0.5 + 0.01 * mk)

    err = _curves(masks, cg, f)
    rows = opat.subset_pattern(err, masks, cg, 5, 3.0, 0x40, 1.0, 8.0)
    # 0x21 (another base) and 0x03 (no base bit) are not candidates of base 0x40
    assert [r["mask"] for r in rows] == [0x45, 0x43, 0x49, 0x46, 0x4A, 0x4C]
    best = rows[0]
    assert best["best_c"] == cg[np.argmin(np.abs(np.log(cg) - math.log(1.5)))]
    assert best["win_frac"] == 1.0 and all(r["win_frac"] == 0.0 for r in rows[1:])
    # the window excludes a lower minimum outside it
    err2 = err.copy()
    err2[1, 0] = 0.0  # mask 0x45 at c = 0.5, outside [1, 8]
    assert opat.subset_pattern(err2, masks, cg, 5, 3.0, 0x40, 1.0, 8.0)[0] == best
    assert opat.subset_pattern(err2, masks, cg, 5, 3.0, 0x40, 0.5, 8.0)[0]["best_k"] == 0


def test_oracle_pattern_crossing_curves_and_missing_values():
    cg = np.linspace(1.0, 3.0, 21)
    masks = [0x43, 0x45, 0x49]
    err = np.vstack([cg, 4.0 - cg, np.full(cg.size, 10.0)])  # 0x43 wins below c = 2
    rows = opat.subset_pattern(err, masks, cg, 5, 3.0, 0x40, 1.0, 3.0)
    by = {r["mask"]: r for r in rows}
    # at c = 2 the two tie and the smaller mask (0x43) takes it: 11 of 21
    assert by[0x43]["win_frac"] == pytest.approx(11 / 21) and by[0x45]["win_frac"] == pytest.approx(10 / 21)
    assert rows[0]["mask"] == 0x43 and rows[0]["best_k"] == 0
    # +inf (coinciding points) or NaN at one c removes that c from the win count
    err[2, 5] = math.inf
    rows = opat.subset_pattern(err, masks, cg, 5, 3.0, 0x40, 1.0, 3.0)
    assert sum(r["win_frac"] for r in rows) == pytest.approx(1.0)
    assert {r["mask"]: r for r in rows}[0x43]["win_frac"] == pytest.approx(10 / 20)
    # a candidate without any finite error comes last with best_k = -1
    err[1, :] = np.nan
    rows = opat.subset_pattern(err, masks, cg, 5, 3.0, 0x40, 1.0, 3.0)
    assert rows[-1]["mask"] == 0x45 and rows[-1]["best_k"] == -1
    assert all(r["win_frac"] == 0.0 for r in rows)


def test_oracle_pattern_validity_rules():
    """|d| = 1 collapses the d-group to {-1, 1}: bits 4 and 7 are not
    candidates; popcount must be alpha - 2."""
    cg = np.geomspace(1.1, 4.0, 8)
    masks = [0x63, 0x65, 0x69, 0x6C, 0x70, 0x61, 0x67, 0xE1]
    err = np.ones((len(masks), cg.size))
    rows = opat.subset_pattern(err, masks, cg, 6, 1.0, 0x60, 1.0, 4.0)
    assert sorted(r["mask"] for r in rows) == [0x63, 0x65, 0x69, 0x6C]


def _lib_rows(wino, err, masks, cg, size, base, lo, hi):
    return wino.wino_subset_pattern(err, masks, cg, size, base, lo, hi)


@pytest.fixture(scope="module")
def lib():
    import paper_2201_10369_gb300 as w
    w.build()
    w.load()
    return w


def test_library_query_equals_oracle_on_random_arrays(lib):
    rng = np.random.default_rng(7)
    masks = np.array([mk for mk in range(256) if bin(mk).count("1") in (3, 4)], dtype=np.uint8)
    for trial in range(60):
        size = [SIZE_D3, SIZE_D1, (2, 2, 3, 0.5), (2, 4, 3, 2.0)][trial % 4]
        nc = int(rng.integers(1, 40))
        cg = np.sort(rng.uniform(0.3, 6.0, nc))
        err = rng.integers(1, 6, (masks.size, nc)).astype(np.float64)  # many ties
        err[rng.random(err.shape) < 0.05] = np.nan
        err[rng.random(err.shape) < 0.05] = np.inf
        base = int(rng.choice([0x00, 0x20, 0x40, 0x60, 0x80, 0x90]))
        lo, hi = sorted(rng.uniform(0.2, 7.0, 2))
        alpha = size[1] + size[2] - 1
        want = opat.subset_pattern(err, masks, cg, alpha, size[3], base, lo, hi)
        got = _lib_rows(lib, err, masks, cg, size, base, lo, hi)
        assert len(got) == min(len(want), 16)
        for g, w in zip(got, want):
            assert g["mask"] == w["mask"] and g["best_k"] == w["best_k"]
            assert g["win_frac"] == w["win_frac"]
            assert (g["best_err"] == w["best_err"]) or (math.isnan(g["best_err"]) and
                                                        math.isnan(w["best_err"]))


def test_library_query_equals_oracle_on_an_oracle_sweep(lib, orc):
    """Both queries on the oracle's sweep of the bases of Tables 5-6 (F(3,3)
    and F(4,3) with the base points 3, -3, 1/2 and the pair 1, -1)."""
    cg = np.geomspace(1.05, 4.0, 24)
    masks = np.array([mk for mk in range(256) if bin(mk).count("1") in (3, 4)], dtype=np.uint8)
    for m in (3, 4):
        for d, bases in ((3.0, (0x40, 0x20)), (2.0, (0x80,)), (1.0, (0x60,))):
            size = (1, m, 3, d)
            err = orc.error_sweep(cg, [size], masks, 200, 0)[0]
            for base in bases:
                want = opat.subset_pattern(err, masks, cg, m + 2, d, base, 1.0, 4.0)
                got = _lib_rows(lib, err, masks, cg, size, base, 1.0, 4.0)
                assert [(g["mask"], g["best_k"], g["best_err"], g["win_frac"]) for g in got] == \
                       [(w["mask"], w["best_k"], w["best_err"], w["win_frac"]) for w in want]
                assert len(got) == math.comb(4, m - bin(base).count("1"))


def test_library_query_validation(lib):
    err = np.ones((2, 3))
    with pytest.raises(lib.WinoError):
        lib.wino_subset_pattern(err, [0x43, 0x45], [1.0, 2.0, 3.0], SIZE_D3, 0x41)
