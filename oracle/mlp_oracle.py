"""FP64 CPU oracle for the learned hit proposal: a 12 -> 64 -> 64 -> 1
perceptron with ReLU activations scoring (candidate, hit) pairs, trained with
binary cross-entropy on logits and Adam.

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU
baseline; the library never imports it.  The paper has no learned component;
the network, its inputs and its training follow the task's specification of
the proposal (12 inputs, two hidden layers of width 64, one logit, top-k of the
in-window hits).

Pins (the CPU tests): the parameter count; BCE against its closed forms;
gradients against central differences; a network reduced to one layer against
logistic regression; Adam's first steps against their closed forms.

Parameter layout (shared with the library's weight buffer, float32 there):
W1 [12][64] (input-major), b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1] --
5,057 values in that order.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 12, 64
SHAPES = (("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 5057


def unflatten(flat):
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.shape == (N_PARAMS,)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(v):
    """Round to float32, then to bfloat16 (8-bit significand, nearest, ties to
    even), returned as float64."""
    u = np.ascontiguousarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def inference_weights(flat):
    """The network the build ranks with: the weights W1, W2 and W3 in
    bfloat16 (the configuration's "BF16 weights"), the biases in float32 (the
    library keeps them so), from the float32 or float64 master weights."""
    p = unflatten(flat)
    for k in ("W1", "W2", "W3"):
        p[k] = bf16(p[k])
    for k in ("b1", "b2", "b3"):
        p[k] = np.asarray(p[k], dtype=np.float32).astype(np.float64)
    return flatten(p)


def init_params(rng):
    """He-normal weights, zero biases."""
    p = {"W1": rng.normal(0, np.sqrt(2.0 / N_IN), (N_IN, N_HID)), "b1": np.zeros(N_HID),
         "W2": rng.normal(0, np.sqrt(2.0 / N_HID), (N_HID, N_HID)), "b2": np.zeros(N_HID),
         "W3": rng.normal(0, np.sqrt(1.0 / N_HID), N_HID), "b3": np.zeros(1)}
    return flatten(p)


def forward(flat, X):
    """Logits [B] and the activations the backward pass needs."""
    p = unflatten(flat)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"] + p["b3"][0]
    return z, (X, a1, h1, a2, h2)


def bce_with_logits(z, y):
    """mean over the batch of -[y log s(z) + (1-y) log(1-s(z))], written stably."""
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def loss(flat, X, y):
    return bce_with_logits(forward(flat, X)[0], y)


def backward(flat, X, y):
    """Gradient of the mean BCE with respect to the flat parameters."""
    p = unflatten(flat)
    z, (X, a1, h1, a2, h2) = forward(flat, X)
    B = len(z)
    dz = (1.0 / (1.0 + np.exp(-z)) - np.asarray(y, dtype=np.float64)) / B
    g = {"W3": h2.T @ dz, "b3": np.array([dz.sum()])}
    dh2 = np.outer(dz, p["W3"]) * (a2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ p["W2"].T) * (a1 > 0)
    g["W1"] = X.T @ dh1
    g["b1"] = dh1.sum(0)
    return flatten(g)


def adam_step(flat, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba): returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
