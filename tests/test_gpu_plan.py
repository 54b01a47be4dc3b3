"""GPU checks of the planned sweep (one persistent launch in a CUDA graph):
every mode reproduces wino_error_sweep bit for bit, random instance lists
match the oracle, and the device-side deadline stops a run with
WINO_ETIMEOUT instead of letting it run unbounded."""
import math

import numpy as np
import pytest

from paper_2201_10369_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_grid():
    cg = np.sort(np.concatenate([inputs.c_grid(40), [1.0]]))
    return cg, inputs.SWEEP_SIZES, inputs.sweep_masks()


@pytest.mark.parametrize("mode", [1, 2, 3, 0])
def test_plan_modes_equal_grid_sweep(wino, small_grid, mode):
    cg, sizes, masks = small_grid
    ref = wino.wino_error_sweep(cg, sizes, masks, 200, seed=3)
    inst = wino.grid_instances(sizes, masks, cg)
    plan = wino.SweepPlan(sizes, inst, 200, seed=3, mode=mode)
    try:
        got = plan.run().reshape(ref.shape)
        got2 = plan.run().reshape(ref.shape)
        info = plan.info()
    finally:
        plan.close()
    assert np.array_equal(got, ref, equal_nan=True)
    assert np.array_equal(got2, ref, equal_nan=True)
    assert info["items"] > 0 and (mode == 0 or info["mode"] == mode)


def test_plan_random_instances_vs_oracle(wino, orc):
    rng = np.random.default_rng(9)
    sizes = inputs.SWEEP_SIZES + [(1, 4, 5, 1.0)]
    masks = inputs.sweep_masks()
    inst = []
    for _ in range(700):
        s = int(rng.integers(len(sizes)))
        inst.append((s, int(rng.choice(masks)), float(np.exp(rng.uniform(np.log(0.05), np.log(20))))))
    inst += [(2, 0x0F, 1.0), (9, 0x0F, 1.0), (0, 0x07, 1.5)]  # coinciding points; invalid mask
    plan = wino.SweepPlan(sizes, inst, 150, seed=5, mode=1)
    try:
        got = plan.run()
    finally:
        plan.close()
    for (s, mk, c), e in zip(inst, got):
        eo = orc.error_sweep([c], [sizes[s]], [mk], 150, 5)[0, 0, 0]
        if math.isnan(eo):
            assert math.isnan(e)
        elif math.isinf(eo):
            assert math.isinf(e)
        else:
            assert abs(e - eo) <= 1e-6 * eo


def test_plan_deadline_reports_timeout(wino):
    cg = inputs.c_grid(256)
    inst = wino.grid_instances([(2, 6, 3, 1.0)], [0x6F], cg)
    plan = wino.SweepPlan([(2, 6, 3, 1.0)], inst, 1000, seed=0, mode=1)
    try:
        plan.set_deadline(1e-6)  # one nanosecond of device time
        with pytest.raises(wino.WinoError) as e:
            plan.run()
        assert e.value.status == wino.WINO_ETIMEOUT
        plan.set_deadline(0.0)   # the plan stays usable afterwards
        full = plan.run()
        assert np.all(np.isfinite(full))
    finally:
        plan.close()


def test_chunk_split_is_bit_identical(wino):
    """A plan large enough to fill the GPU runs every trial of an instance in
    one lane; a small plan spreads each instance's 128-trial chunks over
    several warps and adds their partial sums afterwards.  Both use the same
    fixed summation order, so the same instance gives the same bits (300
    trials: two full chunks and a ragged one)."""
    sizes = [(1, 2, 3, 1.0)]
    masks = np.array(wino.valid_masks(sizes[0], inputs.sweep_masks()), dtype=np.uint8)
    rng = np.random.default_rng(21)
    n = 32 * 152 * 8 * 4 + 77  # more groups of 32 than four rounds of resident warps
    inst = wino.instance_array(np.zeros(n, np.int32), masks[rng.integers(masks.size, size=n)],
                               np.exp(rng.uniform(np.log(0.05), np.log(20), n)))
    big = wino.SweepPlan(sizes, inst, 300, seed=4, mode=1)
    sub = inst[rng.choice(n, 500, replace=False)]
    small = wino.SweepPlan(sizes, sub, 300, seed=4, mode=1)
    try:
        want = big.run()
        got = small.run()
    finally:
        big.close()
        small.close()
    key = {(int(q["mask"]), float(q["c"])): e for q, e in zip(inst, want)}
    assert np.array_equal(got, np.array([key[(int(q["mask"]), float(q["c"]))] for q in sub]))


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_mixed_split_and_whole_sizes(wino, mode):
    """Chunks are split per size: in one plan a size with more groups of 32
    than four rounds of resident warps runs whole trials per lane while a
    small size spreads its chunks over several items, and only the small
    size's partial sums are combined.  Each instance must give the bits it
    gives in a plan of its size alone (a whole plan for the large size, a
    split one for the small size), in every execution mode."""
    big_size, small_size = (1, 2, 3, 1.0), (2, 6, 3, 1.0)
    rng = np.random.default_rng(33)
    mb = np.array(wino.valid_masks(big_size, inputs.sweep_masks()), dtype=np.uint8)
    ms = np.array(wino.valid_masks(small_size, inputs.sweep_masks()), dtype=np.uint8)
    nb, ns = 32 * 152 * 8 * 4 + 77, 900
    cb = np.exp(rng.uniform(np.log(0.05), np.log(20), nb))
    cs = np.exp(rng.uniform(np.log(0.05), np.log(20), ns))
    inst_b = wino.instance_array(np.zeros(nb, np.int32), mb[rng.integers(mb.size, size=nb)], cb)
    inst_s = wino.instance_array(np.zeros(ns, np.int32), ms[rng.integers(ms.size, size=ns)], cs)
    both = wino.instance_array(np.concatenate([np.zeros(ns, np.int32), np.ones(nb, np.int32)]),
                               np.concatenate([inst_s["mask"], inst_b["mask"]]),
                               np.concatenate([cs, cb]))
    plans = [wino.SweepPlan([big_size], inst_b, 300, seed=8, mode=1),
             wino.SweepPlan([small_size], inst_s, 300, seed=8, mode=1),
             wino.SweepPlan([small_size, big_size], both, 300, seed=8, mode=mode)]
    try:
        want_b, want_s, got = (p.run() for p in plans)
    finally:
        for p in plans:
            p.close()
    assert np.array_equal(got[:ns], want_s, equal_nan=True)
    assert np.array_equal(got[ns:], want_b, equal_nan=True)
