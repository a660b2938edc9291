"""CPU FP64 reference of the autotuner's cost-model network.

TEST INFRASTRUCTURE ONLY (see the package docstring): the tests compare the GPU forward
and backward kernels of the cost model against these plain numpy functions.

Network: two tanh hidden layers of H units, F inputs, one linear output,
    a1 = tanh(W1 x + b1),  a2 = tanh(W2 a1 + b2),  f(x) = w3 . a2 + b3,
loss L = (1/n) sum_s (f(x_s) - y_s)^2, parameters flattened in the order
W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
Parity status: pinned by central finite differences of the loss (tests/test_costmodel_oracle.py).
"""
from __future__ import annotations

import numpy as np


def unpack(p, F, H):
    p = np.asarray(p, np.float64)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]; o += 1
    assert o == p.size
    return W1, b1, W2, b2, w3, b3


def forward(p, X, F, H):
    W1, b1, W2, b2, w3, b3 = unpack(p, F, H)
    X = np.asarray(X, np.float64)
    a1 = np.tanh(X @ W1.T + b1)
    a2 = np.tanh(a1 @ W2.T + b2)
    return a2 @ w3 + b3, a1, a2


def loss(p, X, y, F, H):
    f, _, _ = forward(p, X, F, H)
    return float(np.mean((f - np.asarray(y, np.float64)) ** 2))


def gradient(p, X, y, F, H):
    """Analytic gradient of the loss by the chain rule, layer by layer."""
    W1, b1, W2, b2, w3, b3 = unpack(p, F, H)
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    f, a1, a2 = forward(p, X, F, H)
    g = 2.0 * (f - np.asarray(y, np.float64)) / n          # dL/df
    d2 = (g[:, None] * w3[None, :]) * (1.0 - a2 ** 2)     # dL/dz2
    d1 = (d2 @ W2) * (1.0 - a1 ** 2)                      # dL/dz1
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    gW2 = d2.T @ a1
    gb2 = d2.sum(0)
    gw3 = a2.T @ g
    gb3 = g.sum()
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def numerical_gradient(p, X, y, F, H, h=1e-6):
    """Central differences of the loss, one parameter at a time."""
    p = np.asarray(p, np.float64).copy()
    out = np.empty_like(p)
    for i in range(p.size):
        old = p[i]
        p[i] = old + h
        lp = loss(p, X, y, F, H)
        p[i] = old - h
        lm = loss(p, X, y, F, H)
        p[i] = old
        out[i] = (lp - lm) / (2 * h)
    return out
