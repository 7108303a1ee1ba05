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


def _hand_network():
    """A network whose every layer is worked out by hand below: three inputs,
    a few non-zero weights per layer, non-zero biases in every layer,
    negative pre-activations that the ReLU must clip, and asymmetric W2 / W3
    entries (a transposed matrix reads different entries)."""
    t = np.zeros(mlp.NPARAM)

    def W(name, o, i, v, n_in):
        t[mlp.OFF[name][0] + o * n_in + i] = v

    def b(name, o, v):
        t[mlp.OFF[name][0] + o] = v

    W('W1', 0, 0, 1.0, 16); W('W1', 0, 1, 1.0, 16); b('b1', 0, 0.5)
    W('W1', 1, 2, 2.0, 16); b('b1', 1, -1.0)
    W('W1', 2, 1, -1.0, 16); b('b1', 2, 0.25)
    W('W2', 3, 1, 1.0, 128); W('W2', 3, 2, 2.0, 128); b('b2', 3, 0.5)
    W('W2', 4, 0, 100.0, 128); W('W2', 4, 1, -1.0, 128); b('b2', 4, 1.0)
    W('W2', 5, 0, -4.0, 128); b('b2', 5, 3.0)
    W('W3', 7, 3, 0.5, 128); W('W3', 7, 5, 1.0, 128); b('b3', 7, -2.0)
    W('W3', 8, 3, -1.0, 128); b('b3', 8, 4.0)
    W('W3', 9, 5, 2.0, 128); b('b3', 9, -1.0)
    W('W3', 10, 4, 0.25, 128)
    b('w4', 7, 0.5); b('w4', 8, 10.0); b('w4', 9, -0.25); b('w4', 10, -2.0); b('b4', 0, -3.0)
    x = np.array([[1.0, -2.0, 3.0], [0.0, 0.0, 0.0]])
    return t, x


def test_forward_hand_worked():
    # row A = (1, -2, 3):
    #   a1 = (1 - 2 + 0.5, 2*3 - 1, 2 + 0.25) = (-0.5, 5, 2.25)      h1 = (0, 5, 2.25)
    #   a2[3..5] = (5 + 4.5 + 0.5, 0 - 5 + 1, 0 + 3) = (10, -4, 3)    h2[3..5] = (10, 0, 3)
    #   a3[7..10] = (5 + 3 - 2, -10 + 4, 6 - 1, 0) = (6, -6, 5, 0)    h3[7..10] = (6, 0, 5, 0)
    #   z = 0.5*6 + 10*0 - 0.25*5 - 2*0 - 3 = -1.25
    # row B = 0: a1 = b1 = (0.5, -1, 0.25), h1 = (0.5, 0, 0.25)
    #   a2[3..5] = (0.5 + 0.5, 50 + 1, -2 + 3) = (1, 51, 1)
    #   a3[7..10] = (0.5 + 1 - 2, -1 + 4, 2 - 1, 0.25*51) = (-0.5, 3, 1, 12.75)
    #   z = 0 + 30 - 0.25 - 25.5 - 3 = 1.25
    t, x = _hand_network()
    z, (xp, a1, h1, a2, h2, a3, h3, _) = mlp.forward(t, x)
    assert np.array_equal(z, [-1.25, 1.25])
    assert np.array_equal(a1[:, :4], [[-0.5, 5.0, 2.25, 0.0], [0.5, -1.0, 0.25, 0.0]])
    assert np.array_equal(h1[:, :4], [[0.0, 5.0, 2.25, 0.0], [0.5, 0.0, 0.25, 0.0]])
    assert np.array_equal(a2[:, 3:6], [[10.0, -4.0, 3.0], [1.0, 51.0, 1.0]])
    assert np.array_equal(h3[:, 7:11], [[6.0, 0.0, 5.0, 0.0], [0.0, 3.0, 1.0, 12.75]])
    assert np.count_nonzero(h3) == 5
    # every value above is a short binary fraction, so BF16 storage changes nothing
    zb, _ = mlp.forward(t, x, bf16=True)
    assert np.array_equal(zb, z)
    # y = (0, 1): both rows cost log(1 + e^-1.25)
    assert abs(mlp.loss(t, x, [0.0, 1.0]) - math.log1p(math.exp(-1.25))) < 1e-15


def test_gradient_hand_worked():
    # s = sigmoid(-1.25); dz = (s - 0, sigmoid(1.25) - 1) / 2 = (s/2, -s/2)
    # d3 = dz w4 [a3 > 0]: row A (d3[7], d3[9]) = (s/4, -s/8); row B (d3[8], d3[9], d3[10]) = (-5s, s/8, s)
    # d2 = (d3 W3) [a2 > 0]: row A d2[3] = s/8, d2[5] = s/4 - s/4 = 0; row B (d2[3], d2[4], d2[5]) = (5s, s/4, s/4)
    # d1 = (d2 W2) [a1 > 0]: row A (d1[1], d1[2]) = (s/8, s/4); row B (d1[0], d1[2]) = (25s - s, 10s)
    t, x = _hand_network()
    s = 1.0 / (1.0 + math.exp(1.25))
    g = mlp.gradient(t, x, [0.0, 1.0])

    def at(name, *ix, n_in=None):
        o = mlp.OFF[name][0]
        return g[o + (ix[0] * n_in + ix[1] if n_in else ix[0])]

    expect = [
        (at('b4', 0), 0.0),
        (at('w4', 7), 3 * s), (at('w4', 9), 0.5 * 5 * s - 0.5 * s), (at('w4', 10), -12.75 * s / 2),
        (at('W3', 7, 3, n_in=128), 2.5 * s), (at('W3', 8, 5, n_in=128), -5 * s),
        (at('b3', 8), -5 * s), (at('b3', 9), 0.0), (at('b3', 7), s / 4),
        (at('W2', 3, 1, n_in=128), 5 * s / 8), (at('W2', 4, 0, n_in=128), s / 8),
        (at('W2', 1, 3, n_in=128), 0.0), (at('b2', 3), s / 8 + 5 * s), (at('b2', 5), s / 4),
        (at('W1', 1, 2, n_in=16), 3 * s / 8), (at('W1', 2, 1, n_in=16), -s / 2),
        (at('W1', 0, 0, n_in=16), 0.0), (at('b1', 0), 24 * s), (at('b1', 2), s / 4 + 10 * s),
    ]
    for got, want in expect:
        assert abs(got - want) <= 1e-15 * max(1.0, abs(want)), (got, want)


def test_bf16_storage_points():
    # one path through the network: x = 1 + 2^-9 (BF16: 1), W1 = 1 + 2^-8 + 2^-10
    # (BF16: 1 + 2^-7), b1 = 2^-10 (FP32, kept); a1 = 1 + 2^-7 + 2^-10, stored
    # h1 = 1 + 2^-7; W2 = W3 = w4 = 1, so z = 1 + 2^-7 with BF16 storage
    t = np.zeros(mlp.NPARAM)
    t[mlp.OFF['W1'][0]] = 1 + 2 ** -8 + 2 ** -10
    t[mlp.OFF['b1'][0]] = 2 ** -10
    t[mlp.OFF['W2'][0]] = 1.0
    t[mlp.OFF['W3'][0]] = 1.0
    t[mlp.OFF['w4'][0]] = 1.0
    x = np.array([[1 + 2 ** -9]])
    zb, _ = mlp.forward(t, x, bf16=True)
    assert zb[0] == 1 + 2 ** -7
    z, _ = mlp.forward(t, x)
    assert z[0] == (1 + 2 ** -8 + 2 ** -10) * (1 + 2 ** -9) + 2 ** -10
    # the delta stored for layer 3 is rounded: dz w4 = (sigmoid(z) - 0) / 1
    gb = mlp.gradient(t, x, [0.0], bf16=True)
    d3 = mlp.bf16_round(1.0 / (1.0 + math.exp(-zb[0])))
    assert gb[mlp.OFF['b3'][0]] == d3
    assert gb[mlp.OFF['W3'][0]] == d3 * (1 + 2 ** -7)
