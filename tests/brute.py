"""Pure-Python brute force for tiny hypergraphs (independent of oracle/ and the CUDA path).

It enumerates every k-node subset, builds the induced sub-hypergraph as a set
of hyperedges (Def. 2), checks connectivity, and canonicalises the pattern as
the lexicographically smallest sorted tuple of sorted position-tuples over all
k! relabelings (Def. 3). Patterns are compared with the oracle's class ids by
decoding the oracle's canonical masks through the mask layout.
"""
from __future__ import annotations

import itertools


def normalise(edges):
    out = set()
    for e in edges:
        s = frozenset(e)
        if len(s) >= 2:
            out.add(s)
    return out


def connected_pattern(nodes, hedges) -> bool:
    nodes = list(nodes)
    comp = {v: v for v in nodes}

    def find(x):
        while comp[x] != x:
            x = comp[x]
        return x

    for e in hedges:
        e = list(e)
        for x in e[1:]:
            a, b = find(e[0]), find(x)
            if a != b:
                comp[b] = a
    return len({find(v) for v in nodes}) == 1


def canonical_pattern(k, hedges_pos):
    """hedges_pos: iterable of tuples of positions 0..k-1."""
    best = None
    for perm in itertools.permutations(range(k)):
        form = tuple(sorted(tuple(sorted(perm[p] for p in e)) for e in hedges_pos))
        if best is None or form < best:
            best = form
    return best


def census(edges, n, k):
    """dict canonical pattern -> count, over connected induced k-node sub-hypergraphs."""
    E = normalise(edges)
    small = [e for e in E if len(e) <= k]
    counts = {}
    for V in itertools.combinations(range(n), k):
        Vs = set(V)
        ind = [e for e in small if e <= Vs]
        if not ind or not connected_pattern(V, ind):
            continue
        pos = {v: i for i, v in enumerate(V)}
        pat = canonical_pattern(k, [tuple(pos[x] for x in e) for e in ind])
        counts[pat] = counts.get(pat, 0) + 1
    return counts


def subsets_layout(k):
    """Mask layout: subsets of positions of size 2..k, by size then lexicographic."""
    out = []
    for s in range(2, k + 1):
        out.extend(itertools.combinations(range(k), s))
    return out


def mask_to_pattern(k, mask):
    lay = subsets_layout(k)
    return [lay[b] for b in range(len(lay)) if (mask >> b) & 1]


def oracle_hist_to_patterns(k, hist, canon_masks):
    out = {}
    for c, v in enumerate(hist):
        if int(v):
            out[canonical_pattern(k, mask_to_pattern(k, int(canon_masks[c])))] = int(v)
    return out
