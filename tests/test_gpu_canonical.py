"""Canonical generation checked directly (hm_debug_canonical_check).

The census does not dedupe with a visited set: its per-candidate families
accept each connected k-node set exactly once, by rules on the set's own
structure. Here every set they accept is emitted as a key, the keys are
radix-sorted, and there must be no repeated key and exactly as many keys as
the oracle's census has sets (stored oracle histograms, or the oracle run
on the spot for tiny graphs).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2209_10241_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("case", ["uniform-200", "f2f-330", "coauth-1m-s001", "coauth-1m-s005",
                                  "comm-5m-s001"])
@pytest.mark.parametrize("k", [3, 4])
def test_each_set_once_on_stored_workloads(hm, case, k):
    path = os.path.join(GOLDEN, f"census_{case}.json")
    if not os.path.exists(path):
        pytest.skip(f"stored oracle histogram {case} not written yet")
    with open(path) as f:
        rec = json.load(f)
    total = sum(rec["hist"][str(k)])
    if total > 6e8:
        pytest.skip("more sets than the check's key buffer is sized for here")
    h = synth.workload(rec["workload"], seed=rec["seed"], scale=rec["scale"])
    g = hm.from_host(h, 4)
    sets, repeats = hm.debug_canonical_check(g, k)
    assert repeats == 0
    assert sets == total


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("k", [3, 4])
def test_each_set_once_on_tiny_graphs(hm, seed, k):
    h = synth.random_tiny(7 + seed % 6, 12 + 4 * seed, max_size=6, seed=900 + seed,
                          dup_frac=0.3)
    g = hm.from_host(h, 4)
    sets, repeats = hm.debug_canonical_check(g, k)
    want = oracle.Graph.from_hypergraph(h, 4).census(k, threads=os.cpu_count() or 1)[0]
    assert repeats == 0 and sets == int(want.sum())
