"""Pins of the configuration-model chain of the oracle (oracle.config_mcmc), CPU only.

* invariants: every degree and every hyperedge size is kept, no hyperedge
  gets a repeated member, zero sweeps return the input;
* the stationary distribution is uniform over the hyperedge-labelled
  hypergraphs with the input's degrees and sizes, which is what the
  configuration model is: on a state space small enough to enumerate (four
  hyperedges on five nodes), the states reached from the input by pairwise
  reshuffles are listed by brute force, and 12,000 independent draws fall on
  them within a chi-square bound of the uniform counts;
* on a larger random hypergraph the draws differ from the input and from
  each other (the chain moves).
"""
import itertools

import numpy as np

import oracle
from paper_2209_10241_gb300 import synth


def _edges(mem, off):
    return [tuple(mem[off[j]:off[j + 1]].tolist()) for j in range(len(off) - 1)]


def test_invariants():
    h = synth.workload("coauth-1m", seed=3, scale=0.002)
    out = oracle.config_mcmc(h.members, h.offsets, seed=7, model=2, sweeps=5)
    n = h.num_nodes
    assert np.array_equal(np.bincount(out, minlength=n), np.bincount(h.members, minlength=n))
    for e in _edges(out, h.offsets):
        assert len(set(e)) == len(e)
    assert not np.array_equal(out, h.members)
    assert np.array_equal(oracle.config_mcmc(h.members, h.offsets, seed=7, model=2, sweeps=0),
                          h.members)
    other = oracle.config_mcmc(h.members, h.offsets, seed=7, model=3, sweeps=5)
    assert not np.array_equal(out, other)


def _state(mem, off):
    return tuple(frozenset(e) for e in _edges(mem, off))


def _moves(state):
    """Every state one pairwise reshuffle away (all pairs, all re-deals)."""
    out = set()
    for i, j in itertools.combinations(range(len(state)), 2):
        e, f = state[i], state[j]
        inter = e & f
        rest = sorted((e | f) - inter)
        for a in itertools.combinations(rest, len(e) - len(inter)):
            ne, nf = inter | frozenset(a), inter | (frozenset(rest) - frozenset(a))
            s = list(state)
            s[i], s[j] = ne, nf
            out.add(tuple(s))
    return out


def test_uniform_over_the_reachable_configurations():
    base = [[0, 1], [1, 2], [3, 4], [0, 2, 3]]
    h = synth.from_edges(base, 5)
    start = _state(h.members, h.offsets)
    reach, todo = {start}, [start]
    while todo:
        for s in _moves(todo.pop()):
            if s not in reach:
                reach.add(s)
                todo.append(s)
    # brute force: the reachable states are exactly the labelled hypergraphs
    # with these sizes and degrees
    deg = np.bincount(h.members, minlength=5)
    allc = set()
    for e1, e2, e3 in itertools.product(itertools.combinations(range(5), 2), repeat=3):
        for e4 in itertools.combinations(range(5), 3):
            d = np.bincount(np.array(e1 + e2 + e3 + e4), minlength=5)
            if np.array_equal(d, deg):
                allc.add(tuple(frozenset(x) for x in (e1, e2, e3, e4)))
    assert reach == allc and len(reach) > 20
    counts = {s: 0 for s in reach}
    N = 12000
    for seed in range(N):
        out = oracle.config_mcmc(h.members, h.offsets, seed=seed, model=0, sweeps=12)
        counts[_state(out, h.offsets)] += 1
    K = len(reach)
    E = N / K
    chi2 = sum((c - E) ** 2 / E for c in counts.values())
    df = K - 1
    assert chi2 < df + 5 * np.sqrt(2 * df), (chi2, df)
