"""CPU reference of the per-hyperedge features and proposal targets (TEST INFRASTRUCTURE ONLY).

Features of hyperedge e (rows E_2, E_3, ..., E_k in ascending order), with
d2 = pair degree, t3 = number of 3-hyperedges through a node:
  0: 1, 1: |e|/4, 2-4: log1p(min/mean/max d2), 5-7: log1p(min/mean/max t3),
  8: log1p(#member pairs that are hyperedges), 9: log1p(the number of sets a
  draw of e enumerates at order k), 10: log1p(sum d2), 11: log1p(sum t3),
  12: log1p(#3-hyperedges other than e sharing at least two nodes with e),
  13: log1p(#3-hyperedges inside e), 14-15: 0.
Features 12-13 are counted directly here, triple by triple.
"""
from __future__ import annotations

import numpy as np


def features(g, k: int) -> np.ndarray:
    n = g.n
    E = {s: g.edges(s) for s in range(2, k + 1)}
    d2 = np.zeros(n, dtype=np.int64)
    for a, b in E[2]:
        d2[a] += 1
        d2[b] += 1
    t3 = np.zeros(n, dtype=np.int64)
    if 3 in E:
        for tri in E[3]:
            t3[tri] += 1
    pairs = set(map(tuple, E[2].tolist()))
    tri = [frozenset(t) for t in E[3].tolist()] if 3 in E else []
    # the 3-hyperedges through each node, to meet every triple sharing a node with e
    through = {}
    for t in tri:
        for v in t:
            through.setdefault(v, []).append(t)
    rows = []
    for s in range(2, k + 1):
        for e in E[s].tolist():
            d = d2[e].astype(np.float64)
            t = t3[e].astype(np.float64)
            npairs = sum(1 for i in range(s) for j in range(i + 1, s) if (e[i], e[j]) in pairs)
            if s == 2:
                L = d.sum() - 2
                work = L if k == 3 else L * (L - 1) / 2
            elif s == 3 and k == 4:
                work = d.sum() + t.sum()
            else:
                work = 1.0
            f = np.zeros(16)
            f[0] = 1.0
            f[1] = s / 4
            f[2:5] = np.log1p([d.min(), d.mean(), d.max()])
            f[5:8] = np.log1p([t.min(), t.mean(), t.max()])
            f[8] = np.log1p(npairs)
            f[9] = np.log1p(work)
            f[10] = np.log1p(d.sum())
            f[11] = np.log1p(t.sum())
            es = frozenset(e)
            near = {u for v in e for u in through.get(v, [])}
            f[12] = np.log1p(sum(1 for u in near if u != es and len(u & es) >= 2))
            f[13] = np.log1p(sum(1 for u in near if u <= es and u != es))
            rows.append(f)
    return np.array(rows).reshape(-1, 16)


def targets(contrib: np.ndarray, exact: np.ndarray, countmax: np.ndarray, eps: float):
    """log(sqrt(sum_c (n_ec / countmax_c / T_c)^2) + eps) per hyperedge."""
    T = exact.astype(np.float64)
    ok = T > 0
    y = np.zeros(contrib.shape, dtype=np.float64)
    y[:, ok] = contrib[:, ok] / countmax[ok] / T[ok]
    return np.log(np.sqrt((y ** 2).sum(axis=1)) + eps)
