"""Plain FP64 CPU oracle of the warm-start network (test infrastructure only).

Multilayer perceptron x -> SiLU(x W_1 + b_1) -> ... -> h W_L + b_L with a
linear output layer, mean-squared-error loss, and its gradients by the
chain rule written out layer by layer.  Parameters use the same flat layout
as the CUDA library: for each layer, the weight matrix stored as W^T
(n_out rows of n_in), then the bias (n_out).  Adam follows Kingma & Ba
(2015) with bias correction.

Pinned by tests/test_oracle_mlp.py against central finite differences.
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def layer_shapes(n_in: int, hidden: int, n_hidden: int, n_out: int):
    dims = [n_in] + [hidden] * n_hidden + [n_out]
    return [(dims[k + 1], dims[k]) for k in range(len(dims) - 1)]  # (rows of W^T, cols)


def n_params(shapes) -> int:
    return sum(r * c + r for r, c in shapes)


def unpack(theta: np.ndarray, shapes):
    out, o = [], 0
    for r, c in shapes:
        Wt = theta[o:o + r * c].reshape(r, c)
        o += r * c
        b = theta[o:o + r]
        o += r
        out.append((Wt, b))
    return out


def forward(theta, shapes, x):
    """Returns (y, cache) with cache = list of (input, pre-activation)."""
    cache = []
    h = np.asarray(x, dtype=np.float64)
    layers = unpack(np.asarray(theta, dtype=np.float64), shapes)
    for k, (Wt, b) in enumerate(layers):
        z = h @ Wt.T + b
        cache.append((h, z))
        h = z if k == len(layers) - 1 else silu(z)
    return h, cache


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def grad_from_output(theta, shapes, x, dy):
    """Gradient of sum(y * dy) with respect to the flat parameters."""
    y, cache = forward(theta, shapes, x)
    layers = unpack(np.asarray(theta, dtype=np.float64), shapes)
    grads = []
    g = np.asarray(dy, dtype=np.float64)
    for k in range(len(layers) - 1, -1, -1):
        Wt, b = layers[k]
        h, z = cache[k]
        if k != len(layers) - 1:
            g = g * silu_grad(z)
        grads.append((g.T @ h, g.sum(axis=0)))
        g = g @ Wt
    flat = []
    for dWt, db in reversed(grads):
        flat.append(dWt.reshape(-1))
        flat.append(db)
    return np.concatenate(flat)


def loss_and_grad(theta, shapes, x, t):
    y, _ = forward(theta, shapes, x)
    dy = 2.0 * (y - t) / y.size
    return mse(y, t), grad_from_output(theta, shapes, x, dy)


def adam_step(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
