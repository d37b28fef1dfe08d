"""Pins of the order-5 sampling oracle (Sec. 6.4; oracle.sample5 / sweep5), CPU only.

* canonical form and connectivity: over the 2^10 pair-only masks there are
  34 classes of 5-node graphs, 21 of them connected (the textbook counts of
  graphs on five unlabelled vertices);
* enumeration, max-cardinality rule and classes: taking every hyperedge once
  (sweep5), the total of class c is countmax_c times its exact count, with the
  exact count from the pure-Python brute force over all 5-node subsets
  (tests/brute.py), on random tiny hypergraphs with repeated members,
  duplicates and hyperedges of 6-7 members;
* the estimator: unbiased within 5 standard errors over 300 seeds.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2209_10241_gb300 import synth
from tests import brute

LAYOUT = brute.subsets_layout(5)  # 26 subsets, by size then lexicographic


def test_class_counts_of_simple_graphs():
    classes, connected = set(), set()
    for m in range(1 << 10):
        c = oracle.canonical5(m)
        classes.add(c)
        if oracle.connected5(m):
            connected.add(c)
    assert len(classes) == 34 and len(connected) == 21


def _brute_counts(h):
    pats = brute.census(h.edges(), h.num_nodes, 5)
    return pats


def _pattern(mask):
    return brute.canonical_pattern(5, brute.mask_to_pattern(5, int(mask)))


def _countmax(mask):
    sizes = [len(LAYOUT[b]) for b in range(26) if (int(mask) >> b) & 1]
    top = max(sizes)
    return sizes.count(top)


@pytest.mark.parametrize("seed", range(8))
def test_sweep_equals_countmax_times_exact(seed):
    h = synth.random_tiny(8 + seed % 3, 14 + 2 * seed, max_size=7, seed=500 + seed, dup_frac=0.2)
    masks, sums = oracle.sweep5(h.members, h.offsets, h.num_nodes)
    got = {}
    for m, v in zip(masks, sums):
        p = _pattern(m)
        assert p not in got
        got[p] = (int(v), _countmax(m))
    want = _brute_counts(h)
    assert set(got) == set(want)
    for p, t in want.items():
        v, cm = got[p]
        assert v == cm * t


def test_unbiased_over_seeds():
    h = synth.random_tiny(9, 26, max_size=5, seed=77, dup_frac=0.0)
    exact = {p: t for p, t in _brute_counts(h).items()}
    S = {2: 40, 3: 40, 4: 40, 5: 40}
    R = 300
    sums = {p: [] for p in exact}
    for r in range(R):
        masks, raw, est = oracle.sample5(h.members, h.offsets, h.num_nodes, S, seed=1000 + r)
        e = {_pattern(m): float(x) for m, x in zip(masks, est)}
        for p in exact:
            sums[p].append(e.get(p, 0.0))
    for p, t in exact.items():
        x = np.array(sums[p])
        se = x.std(ddof=1) / np.sqrt(R)
        assert abs(x.mean() - t) <= 5 * se + 1e-9, (p, x.mean(), t, se)
