"""The counting identity behind the sampler's order-4 pair stratum, checked on
the CPU against brute force on small random hypergraphs.

For a drawn pair e = {a, b}, Alg. 4 counts the 4-node sets V' containing e
whose induced sub-hypergraph is connected and holds no 3- or 4-hyperedge.
With N_a = N(a) \\ {b}, N_b = N(b) \\ {a}, T = N_a & N_b, A = N_a - T,
B = N_b - T (sizes sa, sb, t), those sets by pattern are
  (1) c, d in A | B | T: C(sa,2) + C(sb,2) stars, sa sb paths,
      (sa + sb) t paws, C(t,2) diamonds, and each pair cd inside A | B | T
      moves one set to the pattern with cd (star -> paw, path -> 4-cycle,
      paw -> diamond, diamond -> 4-clique);
  (2) c in A | B | T, d a pair neighbour of c outside A | B | T | {a, b}:
      a path, or a paw when c is in T;
less every such set that holds a 3- or 4-hyperedge, each subtracted once:
from a 3-hyperedge {a, b, c} (every d, unless {a, b, d} is one too and
d < c), else from {a, x, y}, else from {b, x, y}, else from the 4-hyperedge.
This restates, in plain Python, the rule the GPU kernels follow, and compares
it with enumerating every 4-node set.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2209_10241_gb300 import synth

PATTERNS = ("star", "path", "paw", "c4", "diamond", "k4")


def _pattern(nodes, pairs):
    """Name of the connected pairs-only pattern on 4 nodes (edge count and
    degree sequence), or None when the pairs do not connect them."""
    edges = [(u, v) for u, v in itertools.combinations(nodes, 2) if frozenset((u, v)) in pairs]
    deg = {v: 0 for v in nodes}
    for u, v in edges:
        deg[u] += 1
        deg[v] += 1
    seen, stack = {nodes[0]}, [nodes[0]]
    while stack:
        x = stack.pop()
        for u, v in edges:
            for p, q in ((u, v), (v, u)):
                if p == x and q not in seen:
                    seen.add(q)
                    stack.append(q)
    if len(seen) < 4:
        return None
    ds = tuple(sorted(deg.values()))
    return {3: "star" if ds == (1, 1, 1, 3) else "path", 4: "paw" if ds == (1, 2, 2, 3) else "c4",
            5: "diamond", 6: "k4"}[len(edges)]


def _brute(a, b, n, pairs, triples, quads):
    out = dict.fromkeys(PATTERNS, 0)
    for c, d in itertools.combinations([x for x in range(n) if x not in (a, b)], 2):
        s = (a, b, c, d)
        if any(frozenset(t) in triples for t in itertools.combinations(s, 3)):
            continue
        if frozenset(s) in quads:
            continue
        p = _pattern(s, pairs)
        if p:
            out[p] += 1
    return out


def _by_types(a, b, adj, pairs, triples, quads, inc3, inc4):
    """The pair stratum's counts for the draw {a, b} by neighbour types."""
    Na, Nb = adj[a] - {b}, adj[b] - {a}
    T, A, B = Na & Nb, Na - Nb, Nb - Na
    ty = {**{x: 0 for x in A}, **{x: 1 for x in B}, **{x: 2 for x in T}}
    sa, sb, t = len(A), len(B), len(T)
    out = dict.fromkeys(PATTERNS, 0)
    out["star"] += sa * (sa - 1) // 2 + sb * (sb - 1) // 2
    out["path"] += sa * sb
    out["paw"] += (sa + sb) * t
    out["diamond"] += t * (t - 1) // 2
    moves = {(0, 0): ("paw", "star"), (1, 1): ("paw", "star"), (0, 1): ("c4", "path"),
             (0, 2): ("diamond", "paw"), (1, 2): ("diamond", "paw"), (2, 2): ("k4", "diamond")}
    for c, tc in ty.items():
        for x in adj[c]:
            if x in (a, b):
                continue
            if x not in ty:
                out["paw" if tc == 2 else "path"] += 1
            elif tc < ty[x] or (tc == ty[x] and c < x):
                up, down = moves[(tc, ty[x])]
                out[up] += 1
                out[down] -= 1

    def has3(*v):
        return frozenset(v) in triples

    def subtract(x, y):
        p = _pattern((a, b, x, y), pairs)
        if p:
            out[p] -= 1

    L1 = set(ty)
    for tri in inc3[a]:
        x, y = sorted(tri - {a})
        if b in (x, y):
            c = y if x == b else x
            for d in (L1 | adj[c]) - {a, b, c}:
                if not (d < c and has3(a, b, d)):
                    subtract(c, d)
        elif not has3(a, b, x) and not has3(a, b, y):
            subtract(x, y)
    for tri in inc3[b]:
        x, y = sorted(tri - {b})
        if a not in (x, y) and not (has3(a, b, x) or has3(a, b, y) or has3(a, x, y)):
            subtract(x, y)
    for q in inc4[a]:
        if b in q:
            x, y = sorted(q - {a, b})
            if not (has3(a, b, x) or has3(a, b, y) or has3(a, x, y) or has3(b, x, y)):
                subtract(x, y)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_counts_by_types_equal_enumeration(seed):
    n = 9 + seed
    h = synth.random_tiny(n, 40 + 12 * seed, max_size=4, seed=500 + seed, dup_frac=0.1)
    g = oracle.Graph.from_hypergraph(h, 4)
    pairs = {frozenset(map(int, e)) for e in g.edges(2)}
    triples = {frozenset(map(int, e)) for e in g.edges(3)}
    quads = {frozenset(map(int, e)) for e in g.edges(4)}
    adj = {v: set() for v in range(n)}
    for e in pairs:
        u, v = tuple(e)
        adj[u].add(v)
        adj[v].add(u)
    inc3 = {v: [t for t in triples if v in t] for v in range(n)}
    inc4 = {v: [q for q in quads if v in q] for v in range(n)}
    assert triples and quads
    for e in pairs:
        a, b = sorted(e)
        want = _brute(a, b, n, pairs, triples, quads)
        got = _by_types(a, b, adj, pairs, triples, quads, inc3, inc4)
        assert got == want, (a, b, got, want)


def test_a_dropped_correction_fails():
    # the same comparison with the 3-hyperedges through both ends ignored
    # must fail on a graph where such sets exist
    pairs = {frozenset(p) for p in [(0, 1), (0, 2), (1, 3), (2, 3), (2, 4)]}
    triples = {frozenset((0, 1, 2))}
    adj = {v: set() for v in range(5)}
    for e in pairs:
        u, v = tuple(e)
        adj[u].add(v)
        adj[v].add(u)
    inc3 = {v: [t for t in triples if v in t] for v in range(5)}
    inc4 = {v: [] for v in range(5)}
    want = _brute(0, 1, 5, pairs, triples, set())
    assert _by_types(0, 1, adj, pairs, triples, set(), inc3, inc4) == want
    assert _by_types(0, 1, adj, pairs, set(), set(), {v: [] for v in range(5)}, inc4) != want
