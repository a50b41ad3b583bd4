"""Multilayer perceptron of the learned Davidson guess (oracle; test infrastructure only).

Fully connected layers h_{l+1} = gelu(W_l h_l + b_l), linear last layer,
gelu(x) = x/2 (1 + erf(x / sqrt 2)); mean-squared-error loss.  Forward and
backward passes written out in float64, to check the GPU training and
inference kernels and (by finite differences) themselves.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

INV_SQRT2 = 1.0 / math.sqrt(2.0)
INV_SQRT2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x * INV_SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x * INV_SQRT2)) + x * INV_SQRT2PI * np.exp(-0.5 * x * x)


def init(sizes, seed):
    """Weights W (out, in) uniform in +-1/sqrt(in), biases zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for fin, fout in zip(sizes[:-1], sizes[1:]):
        lim = 1.0 / math.sqrt(fin)
        params.append((rng.uniform(-lim, lim, size=(fout, fin)), np.zeros(fout)))
    return params


def forward(params, X):
    """Returns the output (N, out) and the per-layer (input, pre-activation) cache."""
    h = np.asarray(X, dtype=np.float64)
    cache = []
    last = len(params) - 1
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if l < last else z
    return h, cache


def loss(Y, T, weights=None):
    """Mean squared error over all entries (optionally weighted per output column)."""
    d = Y - T
    if weights is not None:
        d = d * np.sqrt(weights)[None, :]
    return float(np.mean(d * d))


def backward(params, cache, Y, T, weights=None):
    """Gradients of ``loss`` with respect to every (W, b)."""
    n = Y.size
    g = 2.0 * (Y - T) / n
    if weights is not None:
        g = g * weights[None, :]
    grads = [None] * len(params)
    last = len(params) - 1
    for l in range(last, -1, -1):
        h, z = cache[l]
        if l < last:
            g = g * gelu_grad(z)
        W, _ = params[l]
        grads[l] = (g.T @ h, g.sum(axis=0))
        g = g @ W
    return grads
