"""Element-wise error bounds for the tensor-core MLP against the float64 reference.

The kernels compute the network of ``oracle/mlp.py`` with the same bf16
rounding points, but accumulate in float32 (tensor-core and reduction order
unspecified). Every other difference follows from that: a float32 sum of m
terms differs from the exact sum by at most gamma * (sum of |terms|), and a
bf16 rounding of a value known only within [a - d, a + d] can land anywhere in
[bf16(a - d), bf16(a + d)] (rounding is monotone), which is exactly bf16(a)
unless a rounding midpoint lies within d of a. Running this analysis through
the forward and backward passes gives, for every output and every gradient
element, a bound that is tight where nothing is near a rounding boundary and
widens only by the proven effect of the roundings that can flip. A gradient
entry whose terms are all small gets a small bound, whatever the largest
entry of its block.

A float32 chain of L sequential additions errs by at most L * 2^-23 of the sum
of its |terms| (2^-23 allows truncation as well as rounding to nearest). The
forward dot products have L = k + 1 (k = 16 or 64 products and the bias);
the sums over rows are split as the kernels split them (mlp.cu): each block
sums its rows in order (at least 128 rows, a multiple of 16, at most 512
blocks), and the blocks' partials are added in block order, so
L = rows per block + blocks + 64 (the in-block tree), doubled for margin.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp

U32 = 2.0 ** -23


def row_chain(n: int) -> int:
    """Longest sequential float32 addition chain of a sum over n rows."""
    rows = max(128, ((-(-n // 512)) + 15) // 16 * 16)
    blocks = -(-n // rows)
    return 2 * (rows + blocks + 64)


def _bf16_spread(a, d):
    """Largest change of bf16(v) over v in [a - d, a + d] (0 where no rounding
    midpoint is within d of a)."""
    c = mlp.bf16(a)
    lo = mlp.bf16(a - d)
    hi = mlp.bf16(a + d)
    return np.maximum(np.abs(lo - c), np.abs(hi - c))


def _relu_bf16_spread(a, d):
    c = mlp.bf16(np.maximum(a, 0.0))
    lo = mlp.bf16(np.maximum(a - d, 0.0))
    hi = mlp.bf16(np.maximum(a + d, 0.0))
    return np.maximum(np.abs(lo - c), np.abs(hi - c))


def bounds(p, X, t):
    """(y_ref, dy_bound, g_ref, g_bound, loss_ref, loss_bound) for parameters p,
    inputs X (n x 16) and targets t: |y - y_ref| <= dy_bound and
    |g - g_ref| <= g_bound hold element by element for any float32
    evaluation of the network with the bf16 rounding points of the kernels."""
    p = np.asarray(p, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    r = mlp.bf16
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p)
    W1b, W2b, w3b = r(W1), r(W2), r(w3)
    n = X.shape[0]
    g16, g64, g1 = 17 * U32, 65 * U32, 2 * U32
    gamma = row_chain(n) * U32
    x = r(X)                                     # exact on both sides
    # ---- forward
    z1 = x @ W1b + b1
    dz1_ = g16 * (np.abs(x) @ np.abs(W1b) + np.abs(b1))
    h1 = r(np.maximum(z1, 0.0))
    dh1 = _relu_bf16_spread(z1, dz1_)
    z2 = h1 @ W2b + b2
    dz2_ = g64 * (np.abs(h1) @ np.abs(W2b) + np.abs(b2)) + dh1 @ np.abs(W2b)
    h2 = r(np.maximum(z2, 0.0))
    dh2 = _relu_bf16_spread(z2, dz2_)
    y = h2 @ w3b + b3
    dy_ = g64 * (np.abs(h2) @ np.abs(w3b) + abs(b3)) + dh2 @ np.abs(w3b)
    # ---- backward
    g = np.zeros(mlp.NPARAM)
    gb = np.zeros(mlp.NPARAM)
    e = 2.0 * (y - t) / n
    de = 2.0 * dy_ / n + g1 * np.abs(e)
    g[mlp.P_B3] = e.sum()
    gb[mlp.P_B3] = de.sum() + gamma * np.abs(e).sum()
    g[mlp.P_W3:mlp.P_B3] = e @ h2
    gb[mlp.P_W3:mlp.P_B3] = (de @ np.abs(h2) + np.abs(e) @ dh2 + de @ dh2
                             + gamma * (np.abs(e) @ np.abs(h2)))
    # dz2 = e w3 where z2 > 0; the sign of z2 is uncertain where |z2| <= dz2_
    on2 = z2 > 0
    amb2 = np.abs(z2) <= dz2_
    d2 = np.outer(e, w3b) * on2
    dd2 = (np.outer(de, np.abs(w3b)) + g1 * np.abs(np.outer(e, w3b))) * (on2 | amb2) \
        + np.abs(np.outer(e, w3b)) * amb2
    g[mlp.P_B2:mlp.P_W3] = d2.sum(axis=0)
    gb[mlp.P_B2:mlp.P_W3] = dd2.sum(axis=0) + gamma * np.abs(d2).sum(axis=0)
    d2b = r(d2)
    dd2b = _bf16_spread(d2, dd2)
    g[mlp.P_W2:mlp.P_B2] = (h1.T @ d2b).reshape(-1)
    gb[mlp.P_W2:mlp.P_B2] = (dh1.T @ np.abs(d2b) + np.abs(h1).T @ dd2b + dh1.T @ dd2b
                             + gamma * (np.abs(h1).T @ np.abs(d2b))).reshape(-1)
    a1 = d2b @ W2b.T
    da1 = dd2b @ np.abs(W2b).T + g64 * (np.abs(d2b) @ np.abs(W2b).T)
    on1 = z1 > 0
    amb1 = np.abs(z1) <= dz1_
    d1 = a1 * on1
    dd1 = da1 * (on1 | amb1) + np.abs(a1) * amb1
    g[mlp.P_B1:mlp.P_W2] = d1.sum(axis=0)
    gb[mlp.P_B1:mlp.P_W2] = dd1.sum(axis=0) + gamma * np.abs(d1).sum(axis=0)
    d1b = r(d1)
    dd1b = _bf16_spread(d1, dd1)
    g[mlp.P_W1:mlp.P_B1] = (x.T @ d1b).reshape(-1)
    gb[mlp.P_W1:mlp.P_B1] = (np.abs(x).T @ dd1b
                             + gamma * (np.abs(x).T @ np.abs(d1b))).reshape(-1)
    res = y - t
    loss = float((res ** 2).sum())
    loss_b = float((2 * np.abs(res) * dy_ + dy_ ** 2).sum() + gamma * loss)
    # float32 representation of the outputs themselves
    dy_ = dy_ + 2.0 ** -23 * np.abs(y)
    gb = gb + 2.0 ** -23 * np.abs(g) + 1e-38
    return y, dy_, g, gb, loss, loss_b + 2.0 ** -23 * loss


def simulate_f32(p, X, t, order_seed: int = 0):
    """A float32 evaluation of the network with the kernels' bf16 rounding
    points (sums taken in float32 in a seeded row order), for checking the
    bounds on the CPU: (y, grad, loss)."""
    rng = np.random.default_rng(order_seed)
    f = np.float32
    r32 = lambda a: mlp.bf16(a).astype(f)  # noqa: E731
    W1, b1, W2, b2, w3, b3 = (np.asarray(a, dtype=f) for a in mlp.unpack(p))
    n = X.shape[0]
    x = r32(X)
    z1 = (x @ r32(W1)).astype(f) + b1
    h1 = r32(np.maximum(z1, 0))
    z2 = (h1 @ r32(W2)).astype(f) + b2
    h2 = r32(np.maximum(z2, 0))
    y = (h2 @ r32(w3)).astype(f) + f(b3)
    e = (f(2.0) * (y - np.asarray(t, dtype=f)) / f(n)).astype(f)
    perm = rng.permutation(n)
    g = np.zeros(mlp.NPARAM, dtype=f)
    g[mlp.P_B3] = np.sum(e[perm], dtype=f)
    g[mlp.P_W3:mlp.P_B3] = (e[perm] @ h2[perm]).astype(f)
    d2 = (np.outer(e, r32(w3)) * (z2 > 0)).astype(f)
    g[mlp.P_B2:mlp.P_W3] = np.sum(d2[perm], axis=0, dtype=f)
    d2b = r32(d2)
    g[mlp.P_W2:mlp.P_B2] = (h1[perm].T @ d2b[perm]).astype(f).reshape(-1)
    a1 = (d2b @ r32(W2).T).astype(f)
    d1 = (a1 * (z1 > 0)).astype(f)
    g[mlp.P_B1:mlp.P_W2] = np.sum(d1[perm], axis=0, dtype=f)
    d1b = r32(d1)
    g[mlp.P_W1:mlp.P_B1] = (x[perm].T @ d1b[perm]).astype(f).reshape(-1)
    loss = np.sum(((y - np.asarray(t, dtype=f)) ** 2)[perm], dtype=f)
    return y.astype(np.float64), g.astype(np.float64), float(loss)
