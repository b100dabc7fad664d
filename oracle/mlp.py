"""FP64 CPU oracle of the learned cost predictor / surrogate network.

TEST INFRASTRUCTURE ONLY (tests/ and the CPU baseline use it; the CUDA path
never does). A plain multilayer perceptron written out in numpy float64:

    z1 = x W1 + b1,  h1 = silu(z1)
    z2 = h1 W2 + b2, h2 = silu(z2)
    z3 = h2 W3 + b3, h3 = silu(z3)
    out = h3 W4 + b4
    loss = mean over batch and outputs of (out - y)^2

silu(z) = z * sigmoid(z). Parameters are one flat vector in the order
W1, b1, W2, b2, W3, b3, W4, b4 with W_l stored row-major [fan_in, fan_out],
the layout the CUDA kernels use. Backward is the chain rule layer by layer;
Adam follows Kingma & Ba (2015), Algorithm 1.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(n_in: int, n_hidden: int, n_out: int, n_layers: int = 3):
    dims = [n_in] + [n_hidden] * n_layers + [n_out]
    return [(dims[i], dims[i + 1]) for i in range(len(dims) - 1)]


def n_params(n_in: int, n_hidden: int, n_out: int, n_layers: int = 3) -> int:
    return sum(a * b + b for a, b in layer_shapes(n_in, n_hidden, n_out, n_layers))


def unpack(theta: np.ndarray, shapes):
    out, o = [], 0
    for a, b in shapes:
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        bias = theta[o:o + b]
        o += b
        out.append((W, bias))
    return out


def init_params(n_in, n_hidden, n_out, seed, n_layers=3) -> np.ndarray:
    """He-style normal initialisation (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in layer_shapes(n_in, n_hidden, n_out, n_layers):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / a), a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts)


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(theta, x, shapes):
    """Returns the output and the per-layer cache (inputs, pre-activations)."""
    layers = unpack(theta, shapes)
    h = x
    cache = []
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        cache.append((h, z))
        h = z * _sig(z) if li < len(layers) - 1 else z
    return h, cache


def loss_and_grad(theta, x, y, shapes):
    """MSE loss (mean over all output entries) and its gradient w.r.t. theta."""
    out, cache = forward(theta, x, shapes)
    layers = unpack(theta, shapes)
    diff = out - y
    loss = float(np.mean(diff * diff))
    g = 2.0 * diff / diff.size
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        h_in, z = cache[li]
        if li < len(layers) - 1:
            s = _sig(z)
            g = g * (s * (1.0 + z * (1.0 - s)))     # d silu / dz
        W, _ = layers[li]
        grads[li] = (h_in.T @ g, g.sum(axis=0))
        g = g @ W.T
    flat = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for gw, gb in grads])
    return loss, flat


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new theta, m, v."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1**t)
    vhat = v / (1 - beta2**t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
