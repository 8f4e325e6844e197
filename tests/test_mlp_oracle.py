"""Pins of the rank-predictor MLP oracle (CPU): the analytic gradient against
central finite differences of the loss, closed forms of special parameter
settings, and the first Adam step in closed form."""
import numpy as np

from oracle import mlp
from paper_2408_17116_gb300 import workloads

NIN, NH = 8, 12


def _data(n=40):
    X, t = workloads.mlp_toy_data(n, NIN)
    p = workloads.mlp_init(NIN, NH).astype(np.float64)
    rng = np.random.default_rng(5)
    p = p + 0.1 * rng.standard_normal(p.size)  # non-zero biases exercise every term
    return X.astype(np.float64), t.astype(np.float64), p


def test_gradient_matches_central_differences():
    X, t, p = _data()
    L, g = mlp.loss_grad(p, X, t, NIN, NH)
    assert abs(L - mlp.loss(p, X, t, NIN, NH)) < 1e-14
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss(p + e, X, t, NIN, NH) - mlp.loss(p - e, X, t, NIN, NH)) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_output_bias_only_network():
    # W2 = b2 = 0 gives h2 = 0 and y = b3: dL/db3 = 2 mean(b3 - t), every other gradient 0
    X, t, p = _data()
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, NIN, NH)
    p0 = mlp.pack(W1, b1, 0 * W2, 0 * b2, w3, 0.3)
    L, g = mlp.loss_grad(p0, X, t, NIN, NH)
    assert abs(L - np.mean((0.3 - t) ** 2)) < 1e-14
    assert abs(g[-1] - 2 * np.mean(0.3 - t)) < 1e-14
    gW1, gb1, gW2, gb2, gw3, _ = mlp.unpack(g, NIN, NH)
    assert np.all(gw3 == 0) and np.all(gW1 == 0) and np.all(gb1 == 0)
    # W2 still receives (e w3)^T h1 since tanh'(0) = 1
    e = 2 * (0.3 - t) / t.size
    h1 = np.tanh(X @ W1.T + b1)
    assert np.allclose(gW2, np.outer(w3, e @ h1), atol=1e-14)


def test_first_adam_step_is_signed_learning_rate():
    # m1 = (1 - b1) g, v1 = (1 - b2) g^2: bias correction gives m/sqrt(v) = sign(g)
    rng = np.random.default_rng(1)
    p = rng.standard_normal(30)
    g = rng.standard_normal(30)
    opt = mlp.Adam(30, lr=0.01)
    p1 = opt.step(p, g)
    assert np.allclose(p1, p - 0.01 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), atol=1e-15)
