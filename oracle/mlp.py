"""FP64 oracle of the learned surrogate -- TEST INFRASTRUCTURE ONLY.

A two-layer perceptron f: R^16 -> R, f(x) = w2 . gelu(W1 x + b1) + b2 with
gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, trained with the mean
squared error and Adam (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8).  It
predicts log10 of the sweep error from a point-set description; the paper
has no surrogate (its Sec. 6.1 observation that the error curve is roughly
smooth motivates it).  Parameters are packed as one vector
[W1 (64 x 16, row-major) | b1 (64) | w2 (64) | b2 (1)] = 1153 values.
Only tests use this module.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID = 16, 64
N_PARAM = N_HID * N_IN + N_HID + N_HID + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + N_HID * N_IN].reshape(N_HID, N_IN)
    o += N_HID * N_IN
    b1 = p[o:o + N_HID]
    o += N_HID
    w2 = p[o:o + N_HID]
    o += N_HID
    b2 = p[o]
    return W1, b1, w2, b2


def gelu(z):
    erf = np.vectorize(math.erf)
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    erf = np.vectorize(math.erf)
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def forward(p, X):
    W1, b1, w2, b2 = unpack(p)
    Z = X @ W1.T + b1
    H = gelu(Z)
    return H @ w2 + b2, (Z, H)


def loss_and_grad(p, X, y):
    """MSE over the batch and its analytic gradient (packed like p)."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    B = X.shape[0]
    W1, b1, w2, b2 = unpack(p)
    out, (Z, H) = forward(p, X)
    r = out - y
    loss = np.mean(r * r)
    dout = 2.0 * r / B
    g_w2 = H.T @ dout
    g_b2 = dout.sum()
    dH = np.outer(dout, w2)
    dZ = dH * gelu_grad(Z)
    g_W1 = dZ.T @ X
    g_b1 = dZ.sum(axis=0)
    return loss, np.concatenate([g_W1.ravel(), g_b1, g_w2, [g_b2]])


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
