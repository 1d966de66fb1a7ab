"""Pins for the MLP oracle: central finite differences of its own loss, a
network whose output is known in closed form, dead-ReLU gradients, and the
closed form of Adam's first step."""
import numpy as np

from oracle import mlp


def data(rows=13, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, mlp.IN))
    T = rng.standard_normal((rows, mlp.OUT))
    M = (rng.random((rows, mlp.OUT)) < 0.7).astype(float)
    return X, T, M


def test_gradient_matches_central_differences():
    p = mlp.init_params(3)
    X, T, M = data()
    _, g = mlp.loss_and_grad(p, X, T, M)
    rng = np.random.default_rng(0)
    idx = rng.choice(mlp.NPARAM, 200, replace=False)
    h = 1e-6
    for q in idx:
        e = np.zeros(mlp.NPARAM)
        e[q] = h
        fd = (mlp.loss(p + e, X, T, M) - mlp.loss(p - e, X, T, M)) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(g[q])), (q, fd, g[q])


def test_closed_form_network():
    # W1 = 0, b1 = 1 -> h1 = 1; W2 = 0, b2 = 2 -> h2 = 2;
    # W3[k, 0] = k, b3 = 0.5 -> y_k = 2k + 0.5 for every input.
    W1 = np.zeros((mlp.H, mlp.IN)); b1 = np.ones(mlp.H)
    W2 = np.zeros((mlp.H, mlp.H)); b2 = 2 * np.ones(mlp.H)
    W3 = np.zeros((mlp.OUT, mlp.H)); W3[:, 0] = np.arange(mlp.OUT); b3 = 0.5 * np.ones(mlp.OUT)
    p = mlp.pack(W1, b1, W2, b2, W3, b3)
    X, _, _ = data(5)
    y, _ = mlp.forward(p, X)
    assert np.array_equal(y, np.tile(2 * np.arange(mlp.OUT) + 0.5, (5, 1)))
    # Loss against t = y + 1 on one masked entry: (1)^2 / 1.
    T = y.copy(); T[2, 3] += 1.0
    M = np.zeros_like(y); M[2, 3] = 1.0
    L, g = mlp.loss_and_grad(p, X, T, M)
    assert L == 1.0
    gW1, gb1, gW2, gb2, gW3, gb3 = mlp.unpack(g)
    # dL/db3_3 = 2 (y - t) = -2 ; dL/dW3[3, j] = -2 * h2_j = -4.
    assert gb3[3] == -2.0 and np.all(gW3[3] == -4.0)


def test_dead_relu_blocks_gradient():
    p = mlp.init_params(4)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    b1[:] = -1e6                      # every first-layer unit is off
    p = mlp.pack(W1, b1, W2, b2, W3, b3)
    X, T, M = data()
    _, g = mlp.loss_and_grad(p, X, T, M)
    gW1, gb1, *_ = mlp.unpack(g)
    assert np.all(gW1 == 0) and np.all(gb1 == 0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    p1, m, v = mlp.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=0.0)
    # With zero moments, step 1 moves every parameter by lr * sign(g).
    assert np.allclose(p1, p - 0.01 * np.sign(g), rtol=0, atol=1e-15)
