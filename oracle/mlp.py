"""Oracle: FP64 reference MLP for the Delta Z surrogate.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The surrogate maps the deposit parameters (6 inputs) to the Delta Z signal
along the probe path (real and imaginary parts, 256 outputs) through four
hidden layers of 256 units.  The activation is unspecified; SiLU is used
(smooth, so finite-difference gradient checks apply).  Loss: mean squared
error L = 1/(2 B D) sum (y - t)^2 over a batch of B samples and D outputs.
Optimiser: Adam (Kingma & Ba) with bias correction.

Layer l computes z_l = x_l W_l^T + b_l with W_l of shape (out, in);
x_{l+1} = silu(z_l) for the hidden layers, y = z_L for the output layer.
"""
from __future__ import annotations

import numpy as np

SIZES = (6, 256, 256, 256, 256, 256)


def sigmoid(z):
    """Logistic function 1/(1 + exp(-z)) (building block of SiLU)."""
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    """SiLU z * sigmoid(z), the hidden activation (reading: the activation is unspecified)."""
    return z * sigmoid(z)


def silu_grad(z):
    """d silu / dz = sigmoid(z) (1 + z (1 - sigmoid(z)))."""
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def init(seed=0, sizes=SIZES):
    """He-style normal init scaled by 1/sqrt(fan_in); zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for i in range(len(sizes) - 1):
        fi, fo = sizes[i], sizes[i + 1]
        W = rng.normal(scale=1.0 / np.sqrt(fi), size=(fo, fi))
        params.append([W, np.zeros(fo)])
    return params


def forward(params, X):
    """Returns (y, cache) with cache = (inputs x_l, pre-activations z_l)."""
    xs, zs = [], []
    x = np.asarray(X, dtype=np.float64)
    L = len(params)
    for l, (W, b) in enumerate(params):
        xs.append(x)
        z = x @ W.T + b
        zs.append(z)
        x = silu(z) if l < L - 1 else z
    return x, (xs, zs)


def loss(y, t):
    """Mean squared error 1/(2 B D) sum (y - t)^2 (module notes)."""
    return 0.5 * np.mean((y - t) ** 2)


def backward(params, cache, y, t):
    """Gradients of loss(y, t) with respect to every (W, b)."""
    xs, zs = cache
    B, D = y.shape
    g = (y - t) / (B * D)                      # dL/dz for the output layer
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        if l < len(params) - 1:
            g = g * silu_grad(zs[l])
        grads[l] = [g.T @ xs[l], g.sum(axis=0)]
        g = g @ W
    return grads


def adam_init(params):
    """Zero first and second moments and step 0 for Adam (Kingma & Ba)."""
    return {"t": 0, "m": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
            "v": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]}


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    state["t"] += 1
    t = state["t"]
    for l in range(len(params)):
        for i in range(2):
            g = grads[l][i]
            m = state["m"][l][i]
            v = state["v"][l][i]
            m *= beta1
            m += (1.0 - beta1) * g
            v *= beta2
            v += (1.0 - beta2) * g * g
            mh = m / (1.0 - beta1 ** t)
            vh = v / (1.0 - beta2 ** t)
            params[l][i] -= lr * mh / (np.sqrt(vh) + eps)
    return params
