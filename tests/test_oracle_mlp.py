"""Pins for the CPU references of the proposal MLP and features (no GPU).

* the analytic backward of the unrounded network equals central finite
  differences of its loss;
* bf16 rounding equals torch's float32 -> bfloat16 conversion (round to
  nearest even), including ties;
* one Adam step follows the published update (Kingma & Ba, 2015);
* the features of a hand-built hypergraph equal values worked out by hand.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import features as F
from oracle import mlp
from paper_2209_10241_gb300 import synth


def _data(seed, n=40):
    st = synth.Stream(seed, 21)
    u = (st.u64(n * 17) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    X = (u[: n * 16].reshape(n, 16) * 3.0)
    X[:, 0] = 1.0
    t = u[n * 16:] * 4.0 - 2.0
    return X, t


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_matches_finite_differences(seed):
    p = mlp.init_params(seed).astype(np.float64)
    X, t = _data(seed)
    g = mlp.backward(p, X, t, rounding=False)
    st = synth.Stream(seed, 22)
    idx = np.concatenate([np.arange(mlp.P_B1, mlp.P_B1 + 4), np.arange(mlp.P_W3, mlp.P_W3 + 4),
                          [mlp.P_B3], (st.u64(40) % np.uint64(mlp.NPARAM)).astype(np.int64)])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss(pp, X, t, False) - mlp.loss(pm, X, t, False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding_matches_torch():
    st = synth.Stream(4, 1)
    bits = (st.u64(4096) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[np.isfinite(x) & (np.abs(x) < 1e30)].astype(np.float64)
    x = np.concatenate([x, [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert (mlp.bf16(x) == want).all()
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0           # tie to even
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6


def test_adam_step_formula():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.1, -0.3, 0.0])
    p1, m1, v1 = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, 1e-2)
    # first step: m_hat = g, v_hat = g^2, update = lr * g / (|g| + eps)
    want = p - 1e-2 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1, want, rtol=0, atol=1e-12)


def test_features_by_hand():
    # pairs 01 02 12 23, triple 012, quad 0123 on 5 nodes
    h = synth.from_edges([[0, 1], [0, 2], [1, 2], [2, 3], [0, 1, 2], [0, 1, 2, 3]], 5)
    g = oracle.Graph.from_hypergraph(h, 4)
    f = F.features(g, 4)
    assert f.shape == (4 + 1 + 1, 16)
    d2 = np.array([2, 2, 3, 1, 0])
    # row 0 = pair (0,1): d2 = (2, 2); t3 = (1, 1); L = 2 + 2 - 2 = 2 -> C(2,2) = 1 set
    r = f[0]
    assert np.allclose(r[:12], [1, 0.5, np.log1p(2), np.log1p(2), np.log1p(2), np.log1p(1),
                                np.log1p(1), np.log1p(1), np.log1p(1), np.log1p(1),
                                np.log1p(4), np.log1p(2)])
    # row 4 = triple (0,1,2): d2 = (2,2,3), t3 = (1,1,1), 3 member pairs, work = 7 + 3
    r = f[4]
    assert np.allclose(r[:12], [1, 0.75, np.log1p(2), np.log1p(7 / 3), np.log1p(3), np.log1p(1),
                                np.log1p(1), np.log1p(1), np.log1p(3), np.log1p(10),
                                np.log1p(7), np.log1p(3)])
    # 3-hyperedges sharing >= 2 nodes / inside: the pair (0,1) meets triple 012; the
    # triple has none besides itself; the quad 0123 holds 012 (one sub-triple)
    assert np.isclose(f[0, 12], np.log1p(1)) and f[0, 13] == 0
    assert f[4, 12] == 0 and f[4, 13] == 0
    assert np.isclose(f[5, 12], np.log1p(1)) and np.isclose(f[5, 13], np.log1p(1))
    assert (f[:, 14:] == 0).all() and d2[3] == 1


def test_overlap_features_brute_force():
    """Features 12-13 against counting over every pair of hyperedges."""
    for seed in range(6):
        h = synth.random_tiny(9, 40, max_size=4, seed=seed)
        g = oracle.Graph.from_hypergraph(h, 4)
        f = F.features(g, 4)
        edges = [tuple(e) for s in (2, 3, 4) for e in g.edges(s).tolist()]
        triples = [set(e) for e in edges if len(e) == 3]
        for r, e in enumerate(edges):
            se = set(e)
            share = sum(1 for t in triples if t != se and len(t & se) >= 2)
            inside = sum(1 for t in triples if t < se)
            assert np.isclose(f[r, 12], np.log1p(share)), (seed, e)
            assert np.isclose(f[r, 13], np.log1p(inside)), (seed, e)


def test_targets_formula():
    contrib = np.array([[2, 0], [0, 3], [1, 1]], dtype=np.uint32)
    exact = np.array([4, 0], dtype=np.uint64)
    cm = np.array([2, 1])
    t = F.targets(contrib, exact, cm, eps=1e-3)
    assert np.allclose(t, np.log([2 / 2 / 4 + 1e-3, 1e-3, 1 / 2 / 4 + 1e-3]))
