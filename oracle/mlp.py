"""Reference surrogate network in FP64 NumPy: forward pass, mean binary
cross-entropy and its gradient, written out layer by layer.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  It follows the
network the library trains (not part of the paper): x in R^16 (zero padded),
three ReLU layers of width 128, a logistic output unit,
loss = mean over rows of  -[y log g + (1 - y) log(1 - g)].

Parameter vector layout (FP32 in the library, FP64 here):
W1[128][16], b1[128], W2[128][128], b2[128], W3[128][128], b3[128], w4[128], b4.

``bf16=True`` evaluates the same formulas with the library's storage
precision applied at the points where the library stores a tensor in BF16
(the network's specification: BF16 weights and activations, wider
accumulation): the hidden weight matrices W1..W3, the inputs x, every
hidden activation h_l after its ReLU and, in the gradient, every
back-propagated delta dL/da_l after its mask.  Everything else (biases, w4,
b4, sums) stays FP64.  With ``bf16=False`` it is the plain FP64 network.
"""
from __future__ import annotations

import numpy as np

IN, H = 16, 128
OFF = {}
_o = 0
for name, size in (('W1', H * IN), ('b1', H), ('W2', H * H), ('b2', H), ('W3', H * H), ('b3', H),
                   ('w4', H), ('b4', 1)):
    OFF[name] = (_o, size)
    _o += size
NPARAM = _o


def bf16_round(a):
    """Round FP32 values to the nearest BF16 (ties to even), as float64."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(a):
    return np.asarray(a, np.float64)


def unpack(theta, bf16=False):
    t = np.asarray(theta, np.float64)
    P = {k: t[o:o + s].copy() for k, (o, s) in OFF.items()}
    rw = bf16_round if bf16 else _ident
    P['W1'] = rw(P['W1']).reshape(H, IN)
    P['W2'] = rw(P['W2']).reshape(H, H)
    P['W3'] = rw(P['W3']).reshape(H, H)
    return P


def pad(x):
    x = np.asarray(x, np.float64)
    out = np.zeros((x.shape[0], IN))
    out[:, :x.shape[1]] = x
    return out


def forward(theta, x, bf16=False):
    """Returns (logits z, cache).  Row r of x is one input; layer l computes
    a_l = W_l h_{l-1} + b_l (h_0 = x) and h_l = max(a_l, 0); z = w4 . h3 + b4."""
    rnd = bf16_round if bf16 else _ident
    P = unpack(theta, bf16)
    x = pad(rnd(np.asarray(x, np.float64)))
    a1 = x @ P['W1'].T + P['b1']
    h1 = rnd(np.maximum(a1, 0.0))
    a2 = h1 @ P['W2'].T + P['b2']
    h2 = rnd(np.maximum(a2, 0.0))
    a3 = h2 @ P['W3'].T + P['b3']
    h3 = rnd(np.maximum(a3, 0.0))
    z = h3 @ P['w4'] + P['b4'][0]
    return z, (x, a1, h1, a2, h2, a3, h3, P)


def loss(theta, x, y, bf16=False):
    z, _ = forward(theta, x, bf16)
    y = np.asarray(y, np.float64)
    # -[y log s(z) + (1-y) log(1 - s(z))] = max(z,0) - z y + log(1 + exp(-|z|))
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def gradient(theta, x, y, bf16=False):
    """Gradient of the mean cross-entropy with respect to theta (layout above)."""
    rnd = bf16_round if bf16 else _ident
    z, (x, a1, h1, a2, h2, a3, h3, P) = forward(theta, x, bf16)
    y = np.asarray(y, np.float64)
    n = x.shape[0]
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n            # d loss / d z
    g = np.zeros(NPARAM)

    def put(name, v):
        o, s = OFF[name]
        g[o:o + s] = np.ravel(v)

    put('w4', h3.T @ dz)
    put('b4', [dz.sum()])
    d3 = rnd(np.outer(dz, P['w4']) * (a3 > 0))          # d loss / d a3
    put('W3', d3.T @ h2)
    put('b3', d3.sum(axis=0))
    d2 = rnd((d3 @ P['W3']) * (a2 > 0))
    put('W2', d2.T @ h1)
    put('b2', d2.sum(axis=0))
    d1 = rnd((d2 @ P['W2']) * (a1 > 0))
    put('W1', d1.T @ x)
    put('b1', d1.sum(axis=0))
    return g
