"""Pins for the oracle's exact census (problem statement, Sec. 3; Alg. 1).

The oracle is checked against things other than itself:
* brute force over all k-subsets in pure Python on tiny random hypergraphs
  with duplicates, repeated members, singletons and oversized hyperedges;
* closed forms on complete graphs, stars, paths, cycles and the complete
  3-uniform hypergraph;
* the failure case of the projection baseline (Fig. 2): a set connected in
  the projection but not in the induced sub-hypergraph is not counted;
* invariance under node relabelling and hyperedge reordering/duplication.
"""
from math import comb

import numpy as np
import pytest

import oracle
from paper_2209_10241_gb300 import synth
from tests import brute


def _census(edges, n, k, kmax=4):
    h = synth.from_edges(edges, n)
    g = oracle.Graph.from_hypergraph(h, kmax)
    hist, _ = g.census(k)
    return hist


def _class_by_mask(k, mask):
    canon, _, _ = oracle.class_info(k)
    return int(np.nonzero(canon == oracle.canonical(k, mask))[0][0])


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("k", [3, 4])
def test_bruteforce_tiny(seed, k):
    n = 7 + seed % 3
    h = synth.random_tiny(n, 10 + 2 * seed, max_size=5, seed=seed, dup_frac=0.2)
    edges = h.edges()
    g = oracle.Graph.from_hypergraph(h, 4)
    hist, _ = g.census(k)
    canon, _, _ = oracle.class_info(k)
    want = brute.census(edges, n, k)
    assert brute.oracle_hist_to_patterns(k, hist, canon) == want
    # normalisation: distinct hyperedges per size, set semantics
    E = brute.normalise(edges)
    for s in (2, 3, 4):
        assert g.count(s) == sum(1 for e in E if len(e) == s)
        assert [tuple(r) for r in g.edges(s).tolist()] == sorted(
            tuple(sorted(e)) for e in E if len(e) == s)


@pytest.mark.parametrize("n", [4, 5, 7, 9])
def test_complete_graph(n):
    edges = [[a, b] for a in range(n) for b in range(a + 1, n)]
    h3, h4 = _census(edges, n, 3), _census(edges, n, 4)
    assert h3[_class_by_mask(3, 0b111)] == comb(n, 3) and h3.sum() == comb(n, 3)
    assert h4[_class_by_mask(4, 0b111111)] == comb(n, 4) and h4.sum() == comb(n, 4)


@pytest.mark.parametrize("n", [3, 5, 8])
def test_star(n):
    edges = [[0, i] for i in range(1, n + 1)]
    h3, h4 = _census(edges, n + 1, 3), _census(edges, n + 1, 4)
    assert h3.sum() == comb(n, 2) and h3[_class_by_mask(3, 0b011)] == comb(n, 2)
    # 3-star: pairs 01, 02, 03
    assert h4.sum() == comb(n, 3) and h4[_class_by_mask(4, 0b000111)] == comb(n, 3)


@pytest.mark.parametrize("n", [4, 6, 10])
def test_path(n):
    edges = [[i, i + 1] for i in range(n - 1)]
    h3, h4 = _census(edges, n, 3), _census(edges, n, 4)
    assert h3.sum() == n - 2
    # path 0-1-2-3: pairs 01, 12, 23
    assert h4.sum() == n - 3 and h4[_class_by_mask(4, 0b101001)] == n - 3


@pytest.mark.parametrize("n", [5, 6, 11])
def test_cycle(n):
    edges = [[i, (i + 1) % n] for i in range(n)]
    h3, h4 = _census(edges, n, 3), _census(edges, n, 4)
    assert h3.sum() == n and h3[_class_by_mask(3, 0b011)] == n
    assert h4.sum() == n and h4[_class_by_mask(4, 0b101001)] == n


def test_four_cycle_is_one_c4():
    h4 = _census([[0, 1], [1, 2], [2, 3], [3, 0]], 4, 4)
    c4 = (1 << 0) | (1 << 2) | (1 << 3) | (1 << 5)      # pairs 01, 03, 12, 23
    assert h4.sum() == 1 and h4[_class_by_mask(4, c4)] == 1
    # the other labelling of a 4-cycle (pairs 02, 03, 12, 13) is the same class
    assert _class_by_mask(4, 0b011110) == _class_by_mask(4, c4)


@pytest.mark.parametrize("n", [4, 5, 7])
def test_complete_three_uniform(n):
    edges = [[a, b, c] for a in range(n) for b in range(a + 1, n) for c in range(b + 1, n)]
    h3, h4 = _census(edges, n, 3), _census(edges, n, 4)
    assert h3.sum() == comb(n, 3) and h3[_class_by_mask(3, 0b1000)] == comb(n, 3)
    four_triples = 0b1111 << 6
    assert h4.sum() == comb(n, 4) and h4[_class_by_mask(4, four_triples)] == comb(n, 4)


def test_projection_failure_case_fig2():
    # Fig. 2: one large hyperedge and nothing else. Any k nodes of it are
    # connected in the projection, but the induced sub-hypergraph is empty.
    assert _census([[0, 1, 2, 3, 4]], 5, 3).sum() == 0
    assert _census([[0, 1, 2, 3, 4]], 5, 4).sum() == 0
    assert _census([[0, 1, 2, 3]], 4, 3).sum() == 0
    assert _census([[0, 1, 2, 3]], 4, 4).sum() == 1
    # a node joined only through a hyperedge that leaves the set
    h = _census([[0, 1], [1, 2, 3]], 4, 3)
    assert h.sum() == 1  # {1,2,3}; {0,1,2} is disconnected inside
    assert h[_class_by_mask(3, 0b1000)] == 1


def test_singletons_and_repeats_are_normalised():
    a = _census([[0, 1], [1, 2], [2, 0, 1]], 3, 3)
    b = _census([[1, 0, 0], [2, 1], [5], [1, 2, 0, 2], [0, 1]], 6, 3)
    assert (a == b).all()


@pytest.mark.parametrize("k", [3, 4])
def test_relabel_and_duplication_invariance(k):
    h = synth.workload("uniform-200")
    g0 = oracle.Graph.from_hypergraph(h, 4)
    base, _ = g0.census(k, threads=4)
    st = synth.Stream(99, 5)
    perm = np.argsort(st.u64(h.num_nodes), kind="stable").astype(np.int32)
    edges = [list(perm[np.asarray(e)]) for e in h.edges()]
    order = np.argsort(st.u64(len(edges)), kind="stable")
    edges = [edges[i][::-1] for i in order] + edges[:300]
    h2 = synth.from_edges(edges, h.num_nodes)
    hist, _ = oracle.Graph.from_hypergraph(h2, 4).census(k, threads=4)
    assert (hist == base).all()


def test_order3_independent_of_kmax():
    h = synth.workload("uniform-200")
    a, _ = oracle.Graph.from_hypergraph(h, 3).census(3)
    b, _ = oracle.Graph.from_hypergraph(h, 4).census(3)
    assert (a == b).all()


def test_root_ranges_partition_the_census():
    h = synth.workload("uniform-200")
    g = oracle.Graph.from_hypergraph(h, 4)
    full, _ = g.census(3)
    parts = sum(g.census(3, roots=(lo, lo + 37))[0] for lo in range(0, 200, 37))
    assert (parts == full).all()
