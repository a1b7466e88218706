"""Pin of the MLP oracle: analytic gradient against central finite
differences of the loss (every parameter group, FP64)."""
import numpy as np

from oracle import mlp_oracle as M


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    F, B = 8, 37
    p = rng.standard_normal(M.param_count(F)) * 0.3
    X = rng.standard_normal((B, F))
    T = rng.standard_normal(B)
    _, g = M.loss_and_grad(p, X, T)
    idx = np.concatenate([np.arange(0, 12), [512, 530, 576, 1000, 4671, 4700, 4735, 4736, 4790, 4800]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (M.loss_and_grad(p + e, X, T)[0] - M.loss_and_grad(p - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_mlp_forward_closed_form():
    F = 8
    p = np.zeros(M.param_count(F))
    W1, b1, W2, b2, w3, b3, _ = M.unpack(p, F)
    # only b3 nonzero: the output is the constant b3
    p[-1] = 0.25
    y, _, _ = M.forward(p, np.ones((3, F)))
    np.testing.assert_allclose(y, 0.25)
