"""Pins for the numpy network reference (no GPU)."""
import numpy as np

from oracle import mlp


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    i, h, o, B = 5, 4, 3, 6
    n = sum(int(np.prod(s)) for s in mlp.shapes(i, h, o))
    p = rng.standard_normal(n) * 0.7
    X = rng.standard_normal((B, i))
    T = (rng.random((B, o)) < 0.4).astype(float)
    loss, g = mlp.loss_and_grads(p, X, T, i, h, o)
    eps = 1e-6
    fd = np.zeros(n)
    for k in range(n):
        e = np.zeros(n)
        e[k] = eps
        fd[k] = (mlp.loss_and_grads(p + e, X, T, i, h, o)[0] - mlp.loss_and_grads(p - e, X, T, i, h, o)[0]) / (2 * eps)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_hand_computed_example():
    # one input, identity-like weights: z3 = relu(relu(x W1 + b1) W2 + b2) W3 + b3
    i = h = o = 1
    p = np.array([2.0, 0.5, 3.0, -1.0, 0.25, 0.1])  # W1 b1 W2 b2 W3 b3
    X = np.array([[1.5]])
    # z1 = 3.5, a1 = 3.5, z2 = 9.5, a2 = 9.5, z3 = 2.475
    f = mlp.forward(p, X, i, h, o)
    assert np.isclose(f["z3"][0, 0], 2.475)
    T = np.array([[1.0]])
    loss, g = mlp.loss_and_grads(p, X, T, i, h, o)
    assert np.isclose(loss, np.log1p(np.exp(-2.475)))
    s = 1.0 / (1.0 + np.exp(-2.475))
    # dL/db3 = s - t, dL/dW3 = a2 (s - t)
    assert np.isclose(g[5], s - 1.0) and np.isclose(g[4], 9.5 * (s - 1.0))
