"""GPU checks of the learned surrogate: the hand-written backward pass
against the FP64 oracle's analytic gradient (at the same BF16-rounded
weights), one Adam step against the oracle's update, the row top-k kernel
against numpy, training progress, and what the network gains: the guided
search comes close to the exhaustive sweep's best error per row while
evaluating a small fraction of the instances, and beats a random search of
the same budget."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2201_10369_gb300 import inputs

pytestmark = pytest.mark.gpu


def _batch(B, seed):
    import torch
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (B, 16)).astype(np.float32)
    y = rng.normal(-6, 1, B).astype(np.float32)
    return X, y, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()


def test_mlp_gradient_vs_oracle(wino):
    model = wino.Surrogate(seed=3)
    try:
        rng = np.random.default_rng(4)
        model.set_params(rng.normal(0, 0.3, wino.MLP_PARAMS).astype(np.float32))
        X, y, Xt, yt = _batch(300, 5)
        loss, g = model.loss_grad(Xt, yt)
        pw = model.params(working=True).astype(np.float64)
        lo, go = omlp.loss_and_grad(pw, X, y)
        assert abs(loss - lo) <= 1e-4 * lo
        assert np.max(np.abs(g - go)) <= 1e-3 * np.max(np.abs(go))
    finally:
        model.close()


def test_mlp_adam_step_vs_oracle(wino):
    model = wino.Surrogate(seed=6)
    try:
        rng = np.random.default_rng(7)
        p0 = rng.normal(0, 0.3, wino.MLP_PARAMS).astype(np.float32)
        model.set_params(p0)
        X, y, Xt, yt = _batch(256, 8)
        pw = model.params(working=True).astype(np.float64)
        _, go = omlp.loss_and_grad(pw, X, y)
        model.train(Xt, yt, batch=256, epochs=1, lr=1e-3)
        p1 = model.params().astype(np.float64)
        want, _, _ = omlp.adam_step(p0.astype(np.float64), go, np.zeros_like(go),
                                    np.zeros_like(go), 1, lr=1e-3)
        # first Adam step: each parameter moves by ~lr against its gradient sign;
        # parameters whose gradient is ~0 may differ in sign, so compare where
        # the oracle gradient is clearly nonzero
        big = np.abs(go) > 1e-4 * np.max(np.abs(go))
        assert np.max(np.abs(p1 - want)[big]) <= 2e-5
    finally:
        model.close()


def test_training_is_deterministic(wino):
    """The batch gradient is summed per block and the blocks' partials are
    added in block order (no atomics), so two runs of the same training --
    same initial weights, data and schedule -- end at the same weights, bit
    for bit (several blocks per batch, several steps and epochs)."""
    X, y, Xt, yt = _batch(4096 * 5, 12)
    out = []
    for _ in range(2):
        model = wino.Surrogate(seed=13)
        try:
            model.set_output_bias(float(y.mean()))
            model.train(Xt, yt, batch=4096, epochs=3, lr=3e-3)
            out.append(model.params())
        finally:
            model.close()
    fresh = wino.Surrogate(seed=13)
    try:
        p0 = fresh.params()
    finally:
        fresh.close()
    assert np.array_equal(out[0], out[1])
    assert not np.array_equal(out[0], p0)  # training moved the weights


def test_topk_rows_vs_numpy(wino):
    import torch
    rng = np.random.default_rng(9)
    v = rng.integers(0, 50, (7, 1000)).astype(np.float32)  # many ties
    v[2, 5] = np.nan
    idx = wino.wino_topk_rows(torch.from_numpy(v).cuda(), 32).cpu().numpy()
    for r in range(v.shape[0]):
        vv = np.where(np.isnan(v[r]), np.inf, v[r])
        want = np.lexsort((np.arange(v.shape[1]), vv))[:32]
        assert np.array_equal(idx[r], want)


def test_surrogate_learns_the_error_surface(wino):
    sizes = [(1, 4, 3, 1.0), (2, 4, 3, 1.0), (2, 3, 3, 1.0)]
    masks = inputs.sweep_masks()
    inst, X, y = wino.surrogate_training_set(sizes, masks, 60000, 200, seed=1)
    model = wino.Surrogate(seed=2)
    try:
        n_train = 49152
        var = float(y[n_train:].var())
        model.set_output_bias(float(y[:n_train].mean()))
        model.train(X[:n_train], y[:n_train], batch=1024, epochs=200, lr=3e-3)
        pred = model.predict(X[n_train:])
        mse = float(((pred - y[n_train:]) ** 2).mean())
        assert mse < 0.25 * var, (mse, var)
    finally:
        model.close()


def _ranks(best, ex, rows):
    """Per row: how many grid points of the exhaustive sweep beat `best`."""
    e = np.where(np.isfinite(ex), ex, np.inf)
    return np.array([(e[s, q] < best[s, q]).sum() for s, q in zip(*np.nonzero(rows))])


@pytest.mark.slow
def test_guided_search_gain(wino):
    """What the network gains.  Trained on sweep labels (the bench's set-up:
    2e6 instances, 1000 trials, 200 epochs), the guided search evaluates at
    most 15% of the 4096-c grid: 193 grid points per row (4.7%) plus the
    whole row for each row whose refined proposals lose to the random probe,
    at most one row in ten (8 of 123 measured).  The error it finds per
    (size, mask) row ranks among the best of the exhaustive sweep's 4096
    values of that row: median rank <= 2, 90th percentile <= 32 (0.8% of the
    grid).  A random search given the same per-row budget -- the method
    without the network -- ranks at least 3x worse at the median and worse at
    the 90th percentile.  (The ratio to the row's exhaustive minimum is a
    poor bar: the errors are noisy between neighbouring c, so the minimum of
    4096 noisy values is biased low; its median is still checked <= 1.01.)"""
    sizes = inputs.SWEEP_SIZES
    masks = inputs.sweep_masks()
    trials = inputs.SWEEP_TRIALS
    inst, X, y = wino.surrogate_training_set(sizes, masks, 2_000_000, trials, seed=11)
    model = wino.Surrogate(seed=12)
    try:
        model.set_output_bias(float(y.mean()))
        model.train(X, y, batch=4096, epochs=200, lr=3e-3)
        cg = inputs.c_grid()
        res = wino.guided_sweep(model, sizes, masks, cg, trials, seed=0)
    finally:
        model.close()
    ex = wino.wino_error_sweep(cg, sizes, masks, trials, seed=0)
    ex = np.where(np.isinf(ex), np.nan, ex)
    rows = np.any(np.isfinite(ex), axis=2)
    exb = np.nanmin(np.where(rows[:, :, None], ex, 1.0), axis=2)
    nr = int(rows.sum())
    assert res["evaluated"] == nr * (64 + 64 + 65) + res["fallback_rows"] * cg.size
    assert res["fallback_rows"] <= nr / 10, res["fallback_rows"]
    assert res["evaluated"] <= 0.15 * nr * cg.size
    assert np.median(res["best_err"][rows] / exb[rows]) <= 1.01
    rk = _ranks(res["best_err"], ex, rows)
    assert np.median(rk) <= 2 and np.percentile(rk, 90) <= 32, (np.median(rk), np.percentile(rk, 90))
    budget = 64 + 64 + 65  # the guided search's per-row evaluations before any fallback
    rr = _ranks(wino.random_search(sizes, masks, cg, trials, budget, seed=0), ex, rows)
    assert 3 * max(np.median(rk), 1) <= np.median(rr), (np.median(rk), np.median(rr))
    assert np.percentile(rk, 90) < np.percentile(rr, 90)
