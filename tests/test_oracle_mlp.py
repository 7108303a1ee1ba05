"""Pins of the oracle's reference network: its analytic gradient against
central finite differences of its loss (FP64), the loss of a zero network
(log 2), and the BF16 rounding helper against exact cases."""
import math

import numpy as np

from oracle import mlp


def _theta(rng, scale=0.2):
    return rng.normal(0.0, scale, mlp.NPARAM)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = _theta(rng)
    x = rng.normal(size=(37, 6))
    y = (rng.random(37) < 0.4).astype(float)
    g = mlp.gradient(theta, x, y)
    idx = np.concatenate([rng.choice(mlp.NPARAM, 60, replace=False),
                          [mlp.OFF['b4'][0], mlp.OFF['w4'][0] + 3, mlp.OFF['W1'][0] + 5]])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss(theta + e, x, y) - mlp.loss(theta - e, x, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_zero_network_loss_is_log2():
    x = np.ones((5, 3))
    y = np.array([0, 1, 0, 1, 1.0])
    theta = np.zeros(mlp.NPARAM)
    assert abs(mlp.loss(theta, x, y) - math.log(2.0)) < 1e-15
    g = mlp.gradient(theta, x, y)
    # only the output bias moves: d/db4 = mean(1/2 - y)
    assert abs(g[mlp.OFF['b4'][0]] - np.mean(0.5 - y)) < 1e-15
    assert np.count_nonzero(g) == 1


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 3.0e38], np.float32)
    r = mlp.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0 + 2 ** -7 or r[1] == 1.0  # halfway: ties to even -> 1.0
    assert r[1] == 1.0
    assert r[2] == 1.0 + 2 ** -6
    assert r[3] == 1.0
    assert r[4] == -2.5
