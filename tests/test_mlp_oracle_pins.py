"""Pins of the FP64 proposal-network oracle: central finite differences of
the loss for every parameter, closed forms of binary cross-entropy, and the
Adam update of its defining equations on a case small enough to write out."""
import math

import numpy as np

from oracle import mlp_oracle as M


def test_parameter_count():
    assert M.N_PARAMS == 12 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 5057


def test_bce_closed_forms():
    assert abs(M.bce_with_logits([0.0], [1.0]) - math.log(2.0)) < 1e-15
    assert abs(M.bce_with_logits([0.0], [0.0]) - math.log(2.0)) < 1e-15
    z = 3.7
    assert abs(M.bce_with_logits([z], [1.0]) - math.log1p(math.exp(-z))) < 1e-15
    assert abs(M.bce_with_logits([z], [0.0]) - (z + math.log1p(math.exp(-z)))) < 1e-14
    assert np.isfinite(M.bce_with_logits([800.0, -800.0], [0.0, 1.0]))


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    flat = M.init_params(rng)
    flat[M.N_IN * 64: M.N_IN * 64 + 64] = rng.normal(0, 0.1, 64)  # non-zero b1
    X = rng.normal(size=(37, M.N_IN))
    y = (rng.random(37) < 0.4).astype(np.float64)
    g = M.backward(flat, X, y)
    h = 1e-6
    scale = 0.1 * np.abs(g).max()  # the difference quotient carries ~1e-10 of rounding
    worst = 0.0
    for i in range(M.N_PARAMS):
        a, b = flat.copy(), flat.copy()
        a[i] += h
        b[i] -= h
        fd = (M.loss(a, X, y) - M.loss(b, X, y)) / (2 * h)
        worst = max(worst, abs(fd - g[i]) / (abs(g[i]) + scale))
    assert worst < 1e-6, worst


def test_single_layer_reduction():
    """With W1 = [I 0], W2 = I (inputs kept positive so ReLU passes them) the
    network is logistic regression on W3[:12]: its gradient is X^T (s - y)/B."""
    rng = np.random.default_rng(1)
    p = {"W1": np.hstack([np.eye(12), np.zeros((12, 52))]), "b1": np.zeros(64), "W2": np.eye(64), "b2": np.zeros(64),
         "W3": np.concatenate([rng.normal(size=12), np.zeros(52)]), "b3": np.array([0.3])}
    flat = M.flatten(p)
    X = rng.random((20, 12)) + 0.1
    y = (rng.random(20) < 0.5).astype(np.float64)
    z = X @ p["W3"][:12] + 0.3
    s = 1.0 / (1.0 + np.exp(-z))
    g = M.unflatten(M.backward(flat, X, y))
    assert np.allclose(g["W3"][:12], X.T @ (s - y) / 20, atol=1e-14)
    assert abs(g["b3"][0] - np.mean(s - y)) < 1e-14


def test_adam_first_steps():
    """Adam's bias correction makes the first step lr * sign(g) (for |g| >> eps)."""
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-5)
