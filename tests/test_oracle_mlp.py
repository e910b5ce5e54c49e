"""Pins for the FP64 surrogate MLP oracle (CPU only)."""
import numpy as np

from oracle import mlp


def test_silu_and_derivative():
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(mlp.silu(z), z / (1 + np.exp(-z)), rtol=1e-15)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.silu_grad(z), fd, rtol=1e-8, atol=1e-10)
    assert mlp.silu(0.0) == 0.0 and mlp.silu_grad(0.0) == 0.5


def test_gradients_match_central_differences():
    sizes = (6, 7, 5, 4)
    p = mlp.init(3, sizes)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(9, 6))
    T = rng.normal(size=(9, 4))
    y, cache = mlp.forward(p, X)
    grads = mlp.backward(p, cache, y, T)
    h = 1e-6
    for l in range(len(p)):
        for i in range(2):
            A = p[l][i]
            it = np.nditer(A, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = A[idx]
                A[idx] = old + h
                lp = mlp.loss(mlp.forward(p, X)[0], T)
                A[idx] = old - h
                lm = mlp.loss(mlp.forward(p, X)[0], T)
                A[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(grads[l][i][idx] - fd) <= 1e-7 * max(1.0, abs(fd)), (l, i, idx)


def test_linear_network_reduces_to_least_squares_gradient():
    # one linear layer: dL/dW = (X W^T - T)^T X / (B D)
    p = mlp.init(0, (3, 2))
    rng = np.random.default_rng(2)
    X = rng.normal(size=(5, 3))
    T = rng.normal(size=(5, 2))
    y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, y, T)
    np.testing.assert_allclose(g[0][0], (X @ p[0][0].T - T).T @ X / 10, rtol=1e-14)


def test_adam_first_step_is_lr_times_sign():
    p = [[np.array([[1.0, -2.0]]), np.array([0.5])]]
    g = [[np.array([[3.0, -0.2]]), np.array([-1e-3])]]
    st = mlp.adam_init(p)
    mlp.adam_step(p, g, st, lr=0.1, eps=0.0)
    np.testing.assert_allclose(p[0][0], [[0.9, -1.9]], rtol=1e-14)
    np.testing.assert_allclose(p[0][1], [0.6], rtol=1e-14)


def test_training_reduces_loss():
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, size=(64, 6))
    T = np.sin(X @ rng.normal(size=(6, 8)))
    p = mlp.init(0, (6, 32, 32, 8))
    st = mlp.adam_init(p)
    l0 = mlp.loss(mlp.forward(p, X)[0], T)
    for _ in range(300):
        y, c = mlp.forward(p, X)
        mlp.adam_step(p, mlp.backward(p, c, y, T), st, lr=3e-3)
    assert mlp.loss(mlp.forward(p, X)[0], T) < 0.1 * l0
