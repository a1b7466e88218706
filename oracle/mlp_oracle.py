"""CPU oracle of the rank-predictor MLP (TEST INFRASTRUCTURE ONLY).

FP64 forward pass and analytic backward pass of the 3-layer network
(F -> 64 -> 64 -> 1, tanh hidden layers, linear output) with the loss
mean((f(x) - t)^2), on the same flat parameter layout as the CUDA library:
W1 (64 x F, row-major), b1 (64), W2 (64 x 64, row-major), b2 (64), w3 (64),
b3 (1).  Pinned by finite differences in tests/test_oracle_mlp.py.
"""
import numpy as np

WIDTH = 64


def unpack(p, F):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + WIDTH * F].reshape(WIDTH, F); o += WIDTH * F
    b1 = p[o:o + WIDTH]; o += WIDTH
    W2 = p[o:o + WIDTH * WIDTH].reshape(WIDTH, WIDTH); o += WIDTH * WIDTH
    b2 = p[o:o + WIDTH]; o += WIDTH
    w3 = p[o:o + WIDTH]; o += WIDTH
    b3 = p[o]; o += 1
    return W1, b1, W2, b2, w3, b3, o


def param_count(F):
    return WIDTH * F + WIDTH + WIDTH * WIDTH + WIDTH + WIDTH + 1


def forward(p, X):
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2, w3, b3, _ = unpack(p, X.shape[1])
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3, h1, h2


def loss_and_grad(p, X, T):
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B, F = X.shape
    W1, b1, W2, b2, w3, b3, _ = unpack(p, F)
    y, h1, h2 = forward(p, X)
    loss = np.mean((y - T) ** 2)
    dy = 2.0 * (y - T) / B                       # dL/dy
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    d2 = np.outer(dy, w3) * (1.0 - h2 ** 2)      # dL/d(pre-activation 2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 ** 2)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, g
