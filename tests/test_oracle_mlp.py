"""Pins of the surrogate's FP64 oracle: GELU against known values of the
normal CDF, the analytic gradient against central finite differences, and
Adam's first step against its closed form (each parameter moves by lr in
the direction opposite to its gradient's sign)."""
import math

import numpy as np

from oracle import mlp


def test_gelu_known_values():
    # Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707, Phi(0) = 1/2
    z = np.array([1.0, -1.0, 0.0, 2.0])
    g = mlp.gelu(z)
    assert abs(g[0] - 0.8413447460685429) < 1e-15
    assert abs(g[1] + 0.15865525393145707) < 1e-15
    assert g[2] == 0.0
    assert abs(g[3] - 2 * 0.9772498680518208) < 1e-15


def test_gelu_grad_finite_difference():
    z = np.linspace(-4, 4, 81)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


def test_loss_grad_finite_difference():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, mlp.N_PARAM)
    X = rng.normal(0, 1, (32, mlp.N_IN))
    y = rng.normal(0, 1, 32)
    loss, g = mlp.loss_and_grad(p, X, y)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAM, 60, replace=False).tolist() + [mlp.N_PARAM - 1]
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss_and_grad(p + e, X, y)[0] - mlp.loss_and_grad(p - e, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    p1, m, v = mlp.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    # bias-corrected m = g, v = g^2 on the first step: update = lr g / (|g| + eps)
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(p - p1, 1e-3 * np.sign(g), atol=1e-9)
