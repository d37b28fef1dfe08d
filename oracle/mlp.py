"""CPU reference of the proposal MLP (TEST INFRASTRUCTURE ONLY), numpy float64.

Architecture 16 -> 64 -> 64 -> 1 with ReLU; parameters packed as
W1[16][64] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3 (W[in][out]).
`rounding=True` applies the bf16 rounding points of the tensor-core kernels
(inputs and weights, h1, h2, and the back-propagated dz2 / dz1 entering the
matrix products); `rounding=False` is the plain real-valued network whose
backward the tests check against finite differences.
"""
from __future__ import annotations

import numpy as np

IN, HID = 16, 64
P_W1, P_B1, P_W2, P_B2, P_W3, P_B3 = 0, 1024, 1088, 5184, 5248, 5312
NPARAM = 5313


def bf16(x):
    """Round to bfloat16 (round to nearest even on the fp32 value)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[P_W1:P_B1].reshape(IN, HID), p[P_B1:P_W2], p[P_W2:P_B2].reshape(HID, HID),
            p[P_B2:P_W3], p[P_W3:P_B3], p[P_B3])


def forward(p, X, rounding=True):
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = r(X)
    z1 = x @ r(W1) + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ r(W2) + b2
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ r(w3) + b3
    return y, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2)


def loss(p, X, t, rounding=True):
    y, _ = forward(p, X, rounding)
    return float(np.mean((y - t) ** 2))


def backward(p, X, t, rounding=True):
    """Gradient of mean((y - t)^2) with respect to the packed parameters."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(p)
    y, c = forward(p, X, rounding)
    n = X.shape[0]
    dy = 2.0 * (y - t) / n
    g = np.zeros(NPARAM)
    g[P_B3] = dy.sum()
    g[P_W3:P_B3] = dy @ c["h2"]
    dz2 = np.outer(dy, r(w3)) * (c["z2"] > 0)
    g[P_B2:P_W3] = dz2.sum(axis=0)
    g[P_W2:P_B2] = (c["h1"].T @ r(dz2)).reshape(-1)
    dh1 = r(dz2) @ r(W2).T
    dz1 = dh1 * (c["z1"] > 0)
    g[P_B1:P_W2] = dz1.sum(axis=0)
    g[P_W1:P_B1] = (c["x"].T @ r(dz1)).reshape(-1)
    return g


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return p, m, v


def init_params(seed: int) -> np.ndarray:
    """The seeded initial weights shared with the GPU tests (input generator)."""
    from paper_2209_10241_gb300 import synth
    return synth.mlp_init_params(seed)
