"""Rank-predictor MLP oracle -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy restatement of the learned ACA-rank predictor the library
trains on the GPU (the paper has no learned component; the network only sizes
and orders the ACA of Sec. III).  Used by the tests to check the CUDA forward,
backward and Adam kernels; the library never imports it.

Network: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3.
Parameter packing: W1 [nh][nin] row-major, b1 [nh], W2 [nh][nh], b2 [nh], w3 [nh], b3.
Loss: L = (1/n) sum_s (y_s - t_s)^2.
Adam: Kingma & Ba, "Adam: a method for stochastic optimization", ICLR 2015, Algorithm 1.
"""
import numpy as np


def n_params(nin, nh):
    return nh * nin + nh + nh * nh + nh + nh + 1


def unpack(p, nin, nh):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + nh * nin].reshape(nh, nin); o += nh * nin
    b1 = p[o:o + nh]; o += nh
    W2 = p[o:o + nh * nh].reshape(nh, nh); o += nh * nh
    b2 = p[o:o + nh]; o += nh
    w3 = p[o:o + nh]; o += nh
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [b3]])


def forward(p, X, nin, nh):
    """y[n] and the hidden activations for inputs X[n][nin]."""
    W1, b1, W2, b2, w3, b3 = unpack(p, nin, nh)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3, h1, h2


def loss(p, X, t, nin, nh):
    y, _, _ = forward(p, X, nin, nh)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def loss_grad(p, X, t, nin, nh):
    """(L, dL/dp) by the chain rule, layer by layer (reverse mode)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, nin, nh)
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = X.shape[0]
    y, h1, h2 = forward(p, X, nin, nh)
    e = 2.0 * (y - t) / n                    # dL/dy
    gw3 = h2.T @ e
    gb3 = e.sum()
    d2 = np.outer(e, w3) * (1.0 - h2 ** 2)   # dL/d(pre-activation of layer 2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 ** 2)         # dL/d(pre-activation of layer 1)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    return float(np.mean((y - t) ** 2)), pack(gW1, gb1, gW2, gb2, gw3, gb3)


class Adam:
    """Adam state for a packed parameter vector."""

    def __init__(self, np_, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(np_)
        self.v = np.zeros(np_)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, p, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return p - self.lr * mh / (np.sqrt(vh) + self.eps)
