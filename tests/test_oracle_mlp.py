"""Pins for the oracle MLP of the learned guess: gelu against its definition
and derivative, and every gradient against central finite differences."""
import math

import numpy as np

from oracle import mlp


def test_gelu_definition_and_derivative():
    x = np.linspace(-4, 4, 41)
    ref = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in x])
    assert np.abs(mlp.gelu(x) - ref).max() < 1e-15
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.abs(mlp.gelu_grad(x) - fd).max() < 1e-8


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = mlp.init([5, 7, 6, 2], seed=3)
    params = [(W, rng.normal(size=b.shape) * 0.1) for W, b in params]
    X = rng.normal(size=(9, 5))
    T = rng.normal(size=(9, 2))
    w = np.array([1.0, 0.3])
    Y, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, Y, T, w)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            gflat = g.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 7)):
                old = flat[idx]
                flat[idx] = old + h
                lp = mlp.loss(mlp.forward(params, X)[0], T, w)
                flat[idx] = old - h
                lm = mlp.loss(mlp.forward(params, X)[0], T, w)
                flat[idx] = old
                assert abs((lp - lm) / (2 * h) - gflat[idx]) < 1e-8 * max(1.0, abs(gflat[idx]))
