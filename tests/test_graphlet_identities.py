"""The graphlet identities behind the pairs-only part of the GPU census, checked
on the CPU against brute force over every 4-node set of small random graphs.

With d = degree, t(e) = triangles through pair e, t(v) = triangles at node v,
T = triangles, K4 = 4-cliques and c(x, z) = common neighbours of a node pair,
the not-necessarily-induced counts
  S3 = sum_v C(d, 3), P3 = sum_{uv} (d(u)-1)(d(v)-1) - 3T, TT = sum_v t(v)(d-2),
  D = sum_e C(t(e), 2), C4 = 1/2 sum_{x<z} C(c(x, z), 2)
give the induced counts of the six connected 4-node patterns:
  k4 = K4, diamond = D - 6 K4, c4 = C4 - D + 3 K4, paw = TT - 4 D + 12 K4,
  star = S3 - paw - 2 diamond - 4 k4,
  path = P3 - 2 paw - 4 c4 - 6 diamond - 12 k4.
"""
import itertools

import numpy as np
import pytest


def _sums(A):
    n = len(A)
    d = A.sum(1)
    A2 = A @ A
    T = int(np.trace(A2 @ A)) // 6
    t_node = np.diag(A2 @ A) // 2
    pairs = [(u, v) for u in range(n) for v in range(u + 1, n) if A[u, v]]
    S3 = sum(int(x) * (int(x) - 1) * (int(x) - 2) // 6 for x in d)
    P3 = sum((int(d[u]) - 1) * (int(d[v]) - 1) for u, v in pairs) - 3 * T
    TT = sum(int(t_node[v]) * (int(d[v]) - 2) for v in range(n) if d[v] >= 2)
    D = sum(int(A2[u, v]) * (int(A2[u, v]) - 1) // 2 for u, v in pairs)
    C4 = sum(int(A2[x, z]) * (int(A2[x, z]) - 1) // 2
             for x in range(n) for z in range(x + 1, n)) // 2
    K4 = sum(1 for q in itertools.combinations(range(n), 4)
             if all(A[a, b] for a, b in itertools.combinations(q, 2)))
    return S3, P3, TT, D, C4, K4


def _induced(A):
    """Induced counts of the six connected 4-node patterns by brute force,
    named by edge count and degree sequence."""
    out = dict(star=0, path=0, paw=0, c4=0, diamond=0, k4=0)
    for q in itertools.combinations(range(len(A)), 4):
        es = [(a, b) for a, b in itertools.combinations(q, 2) if A[a, b]]
        deg = sorted(sum(1 for e in es if v in e) for v in q)
        m = len(es)
        if m == 3 and deg == [1, 1, 1, 3]:
            out["star"] += 1
        elif m == 3 and deg == [1, 1, 2, 2]:
            out["path"] += 1
        elif m == 4 and deg == [1, 2, 2, 3]:
            out["paw"] += 1
        elif m == 4 and deg == [2, 2, 2, 2]:
            out["c4"] += 1
        elif m == 5:
            out["diamond"] += 1
        elif m == 6:
            out["k4"] += 1
    return out


@pytest.mark.parametrize("seed", range(12))
def test_identities_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 6 + seed % 5
    A = np.triu((rng.random((n, n)) < 0.25 + 0.05 * (seed % 8)).astype(np.int64), 1)
    A = A + A.T
    S3, P3, TT, D, C4, K4 = _sums(A)
    k4 = K4
    diamond = D - 6 * K4
    c4 = C4 - D + 3 * K4
    paw = TT - 4 * D + 12 * K4
    star = S3 - paw - 2 * diamond - 4 * k4
    path = P3 - 2 * paw - 4 * c4 - 6 * diamond - 12 * k4
    assert dict(star=star, path=path, paw=paw, c4=c4, diamond=diamond, k4=k4) == _induced(A)
