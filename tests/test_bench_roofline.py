"""The bench's algorithmic operation count for the graphlet pair kernel, against
a direct loop over pairs and their common neighbours (CPU only)."""
import numpy as np

import bench


def _brute(e2, n, bw):
    adj = [set() for _ in range(n)]
    for u, v in e2:
        adj[u].add(v)
        adj[v].add(u)
    ops = 0
    for u, v in e2:
        ops += 3 * bw
        for w in adj[u] & adj[v]:
            if w > v:
                ops += 4 * (bw - w // 32)
    return ops


def test_k4_by_hand():
    # 6 pairs x 3 x 4 words, plus the common neighbours above v: (0,1) -> 2, 3;
    # (0,2) -> 3; (1,2) -> 3; four of them x 4 ops x 4 words
    e2 = np.array([[0, 1], [0, 2], [1, 2], [0, 3], [1, 3], [2, 3]])
    assert bench.graphlet_pair_ops(e2, 4, 4) == 72 + 64


def test_random_graphs_match_direct_count():
    rng = np.random.default_rng(3)
    for n in (5, 40, 130):
        bw = ((n + 127) // 128) * 4
        pairs = {tuple(sorted(rng.choice(n, 2, replace=False))) for _ in range(3 * n)}
        e2 = np.array(sorted(pairs))
        assert bench.graphlet_pair_ops(e2, n, bw) == _brute(e2, n, bw)
