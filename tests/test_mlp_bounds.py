"""The element-wise MLP error bounds (tests/mlp_bounds.py) on the CPU.

A float32 evaluation of the network with the kernels' bf16 rounding points
stays inside the bounds of the float64 reference, element by element; a
planted mistake in the float32 evaluation -- a small gradient entry off by
half its value, which the earlier block-scaled tolerance (5e-3 of the
block's largest entry) let through -- falls outside them.
"""
import numpy as np
import pytest

from oracle import mlp
from tests import mlp_bounds
from paper_2209_10241_gb300 import synth


def _data(n, seed):
    st = synth.Stream(seed, 23)
    u = (st.u64(n * 17) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    X = (u[: n * 16].reshape(n, 16) * 4.0).astype(np.float32)
    X[:, 0] = 1.0
    X[:, 12:] = 0.0
    t = (u[n * 16:] * 4.0 - 2.0).astype(np.float32)
    return X, t


@pytest.mark.parametrize("n,seed", [(1, 1), (17, 2), (1000, 3), (5000, 4)])
def test_float32_evaluation_within_bounds(n, seed):
    p = mlp.init_params(seed)
    X, t = _data(n, seed)
    y_ref, yb, g_ref, gb, L, Lb = mlp_bounds.bounds(p, X, t)
    for order_seed in range(3):
        y, g, loss = mlp_bounds.simulate_f32(p, X, t, order_seed)
        assert (np.abs(y - y_ref) <= yb).all()
        assert (np.abs(g - g_ref) <= gb).all()
        assert abs(loss - L) <= Lb


def test_bounds_are_element_wise():
    p = mlp.init_params(5)
    X, t = _data(2000, 6)
    _, _, g_ref, gb, _, _ = mlp_bounds.bounds(p, X, t)
    _, g, _ = mlp_bounds.simulate_f32(p, X, t)
    blocks = [(mlp.P_W1, mlp.P_B1), (mlp.P_B1, mlp.P_W2), (mlp.P_W2, mlp.P_B2),
              (mlp.P_B2, mlp.P_W3), (mlp.P_W3, mlp.P_B3)]
    planted = 0
    for lo, hi in blocks:
        scale = np.abs(g_ref[lo:hi]).max()
        # small entries the block-scaled tolerance would accept at 50 % error
        small = np.where((np.abs(g_ref[lo:hi]) > 0) &
                         (0.5 * np.abs(g_ref[lo:hi]) < 5e-3 * scale) &
                         (gb[lo:hi] < 0.25 * np.abs(g_ref[lo:hi])))[0]
        for i in small[:5]:
            bad = g.copy()
            bad[lo + i] *= 1.5
            assert np.abs(bad[lo + i] - g_ref[lo + i]) > gb[lo + i]
            planted += 1
    assert planted >= 10


def test_dropped_bias_is_caught():
    p = mlp.init_params(7).copy()
    st = synth.Stream(7, 5)
    nb = mlp.P_W2 - mlp.P_B1
    p[mlp.P_B1:mlp.P_W2] = ((st.u64(nb) >> np.uint64(40)).astype(np.float64) / 2 ** 24 - 0.5)
    p[mlp.P_B2:mlp.P_W3] = ((st.u64(nb) >> np.uint64(40)).astype(np.float64) / 2 ** 24 - 0.5)
    X, t = _data(300, 8)
    y_ref, yb, _, _, _, _ = mlp_bounds.bounds(p, X, t)
    q = p.copy()
    q[mlp.P_B2:mlp.P_W3] = 0.0  # a kernel that forgot the second bias
    y, _, _ = mlp_bounds.simulate_f32(q, X, t)
    assert (np.abs(y - y_ref) > yb).any()
