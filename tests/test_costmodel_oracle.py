"""The cost-model reference network's analytic gradient equals central differences."""
import numpy as np

from oracle import mlp


def test_analytic_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    F, H, n = 5, 7, 23
    P = H * F + H + H * H + H + H + 1
    p = rng.standard_normal(P) * 0.5
    X = rng.standard_normal((n, F))
    y = rng.standard_normal(n)
    g = mlp.gradient(p, X, y, F, H)
    gn = mlp.numerical_gradient(p, X, y, F, H)
    assert np.abs(g - gn).max() < 1e-7 * max(1.0, np.abs(gn).max())


def test_linear_limit():
    """With tiny first-layer weights tanh is the identity to first order: f is affine in x."""
    rng = np.random.default_rng(1)
    F, H = 3, 4
    P = H * F + H + H * H + H + H + 1
    p = np.zeros(P)
    p[:H * F] = rng.standard_normal(H * F) * 1e-6
    o = H * F + H
    p[o:o + H * H] = np.eye(H).ravel()
    p[-H - 1:-1] = 1.0
    p[-1] = 0.25
    X = rng.standard_normal((6, F))
    f, _, _ = mlp.forward(p, X, F, H)
    # to first order: a1 = W1 x, a2 = tanh(a1) = a1, f = sum_j a1_j + b3
    lin = X @ p[:H * F].reshape(H, F).sum(0) + 0.25
    assert np.allclose(f, lin, atol=1e-11)
