"""Pins for the oracle's isomorphism classes (Sec. 4.3) against counts fixed by mathematics.

* order 3 has 6 connected patterns (printed in Sec. 4.3);
* Burnside's lemma, computed here from cycle structure, fixes the number of
  all and of connected orbits (8 / 6 for k=3, 180 / 171 for k=4);
* the pairwise-only connected classes are the connected simple graphs on 3
  and 4 nodes (2 and 6, textbook);
* the oracle's class map agrees with an independent pure-Python
  canonicalisation on every labelled pattern.
"""
import itertools

import pytest

import oracle
from tests import brute


def _relabel_python(k, mask, perm):
    lay = brute.subsets_layout(k)
    idx = {t: b for b, t in enumerate(lay)}
    out = 0
    for b, t in enumerate(lay):
        if (mask >> b) & 1:
            out |= 1 << idx[tuple(sorted(perm[p] for p in t))]
    return out


def _connected_python(k, mask):
    return brute.connected_pattern(range(k), [set(t) for t in brute.mask_to_pattern(k, mask)])


@pytest.mark.parametrize("k,total,conn,labelled_conn", [(3, 8, 6, 12), (4, 180, 171, 1990)])
def test_burnside_orbit_counts(k, total, conn, labelled_conn):
    nsub = len(brute.subsets_layout(k))
    perms = list(itertools.permutations(range(k)))
    fix_all = 0
    fix_conn = 0
    conn_masks = [m for m in range(1 << nsub) if _connected_python(k, m)]
    for p in perms:
        # orbits of p on the subset set: fixed patterns are unions of cycles
        lay = brute.subsets_layout(k)
        seen, cycles = set(), 0
        for t in lay:
            if t in seen:
                continue
            cycles += 1
            cur = t
            while cur not in seen:
                seen.add(cur)
                cur = tuple(sorted(p[x] for x in cur))
        fix_all += 2 ** cycles
        fix_conn += sum(1 for m in conn_masks if _relabel_python(k, m, p) == m)
    assert fix_all % len(perms) == 0 and fix_conn % len(perms) == 0
    assert fix_all // len(perms) == total
    assert fix_conn // len(perms) == conn
    assert len(conn_masks) == labelled_conn
    assert oracle.num_classes(k) == conn


def test_order3_has_six_motifs():
    # Sec. 4.3 states that three nodes admit six patterns
    assert oracle.num_classes(3) == 6


@pytest.mark.parametrize("k,expected", [(3, 2), (4, 6)])
def test_pairwise_only_classes_are_connected_simple_graphs(k, expected):
    canon, _, _ = oracle.class_info(k)
    pair_bits = (1 << (k * (k - 1) // 2)) - 1
    assert sum(1 for c in canon if int(c) & ~pair_bits == 0) == expected


@pytest.mark.parametrize("k", [3, 4])
def test_class_map_matches_python_canonicalisation(k):
    nsub = len(brute.subsets_layout(k))
    canon, _, _ = oracle.class_info(k)
    canon_form = {brute.canonical_pattern(k, brute.mask_to_pattern(k, int(c))): i
                  for i, c in enumerate(canon)}
    assert len(canon_form) == len(canon)   # distinct classes are distinct patterns
    for m in range(1 << nsub):
        c = oracle.class_of(k, m)
        if not _connected_python(k, m):
            assert c == -1
            continue
        assert c == canon_form[brute.canonical_pattern(k, brute.mask_to_pattern(k, m))]


@pytest.mark.parametrize("k", [3, 4])
def test_class_ids_are_ranks_of_canonical_masks(k):
    canon, _, _ = oracle.class_info(k)
    assert list(canon) == sorted(canon)
    nsub = len(brute.subsets_layout(k))
    for c in canon:
        # the canonical mask is the minimum over its orbit
        orbit = {_relabel_python(k, int(c), p) for p in itertools.permutations(range(k))}
        assert int(c) == min(orbit)
        assert oracle.canonical(k, max(orbit)) == int(c)
    assert all(int(c) < (1 << nsub) for c in canon)


@pytest.mark.parametrize("k", [3, 4])
def test_maxcard_countmax_from_patterns(k):
    canon, mc, cm = oracle.class_info(k)
    for c, a, b in zip(canon, mc, cm):
        sizes = [len(t) for t in brute.mask_to_pattern(k, int(c))]
        assert a == max(sizes)
        assert b == sizes.count(max(sizes))
    if k == 3:
        got = sorted(zip(mc.tolist(), cm.tolist()))
        # wedge, triangle, and the four patterns holding the 3-hyperedge
        assert got == [(2, 2), (2, 3), (3, 1), (3, 1), (3, 1), (3, 1)]
    else:
        # with the 4-hyperedge present every pattern of the other 10 subsets is
        # connected, so the maxcard-4 classes are the orbits of those patterns
        lay = [t for t in brute.subsets_layout(4) if len(t) < 4]
        fix = 0
        perms = list(itertools.permutations(range(4)))
        for p in perms:
            seen, cycles = set(), 0
            for t in lay:
                if t in seen:
                    continue
                cycles += 1
                cur = t
                while cur not in seen:
                    seen.add(cur)
                    cur = tuple(sorted(p[x] for x in cur))
            fix += 2 ** cycles
        assert sum(1 for a in mc if a == 4) == fix // len(perms)
