"""Pins of the FP64 network oracle: central finite differences of the loss
against the analytic gradient, and closed forms of the cross-entropy."""
import math

import numpy as np

from oracle import mlp


def test_finite_differences_small_network():
    f, h, c = 5, 7, 4
    rng = np.random.default_rng(0)
    w = rng.normal(size=mlp.param_count(f, h, c)) * 0.7
    X = rng.normal(size=(9, f))
    y = rng.integers(0, c, size=9)
    L, g = mlp.loss_grad(w, X, y, f, h, c)
    assert math.isclose(L, mlp.loss(w, X, y, f, h, c), rel_tol=1e-12)
    eps = 1e-6
    num = np.zeros_like(w)
    for i in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        num[i] = (mlp.loss(wp, X, y, f, h, c) - mlp.loss(wm, X, y, f, h, c)) / (2 * eps)
    assert np.max(np.abs(num - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_cross_entropy_closed_forms():
    f, h, c = 3, 4, 6
    w = np.zeros(mlp.param_count(f, h, c))  # all logits 0: loss = log C, softmax uniform
    X = np.ones((5, f))
    y = np.array([0, 1, 2, 3, 5])
    L, g = mlp.loss_grad(w, X, y, f, h, c)
    assert math.isclose(L, math.log(c), rel_tol=1e-14)
    # with W3 = 0 the bias gradient is mean(softmax - onehot): uniform minus label frequencies
    gb3 = g[-c:]
    want = np.full(c, 1.0 / c) - np.bincount(y, minlength=c) / len(y)
    assert np.allclose(gb3, want, atol=1e-15)
    assert abs(gb3.sum()) < 1e-15
