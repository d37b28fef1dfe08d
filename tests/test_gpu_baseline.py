"""The Alg. 1 baseline on the GPU (hm_count_exact_baseline) against the oracle.

Its histogram must equal the exact census bit for bit: tiny random
hypergraphs with repeated members, duplicates and hyperedges larger than k
(which join nodes in the projection without lying inside any k-set), the
Fig. 2 case, and the stored oracle histograms of two workloads. Its
candidate count must equal the closed form on the projection's degrees
(sum C(d, 2) for k = 3; sum C(d, 3) + sum over pairs (d(u) - 1)(d(v) - 1) for
k = 4), computed here from the raw hyperedges.
"""
import itertools
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2209_10241_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _projection(h):
    pairs = set()
    for e in h.edges():
        for a, b in itertools.combinations(sorted(set(e)), 2):
            pairs.add((a, b))
    d = np.zeros(h.num_nodes, dtype=np.int64)
    for a, b in pairs:
        d[a] += 1
        d[b] += 1
    return pairs, d


def _closed_form(h, k):
    pairs, d = _projection(h)
    if k == 3:
        return int(sum(x * (x - 1) // 2 for x in d)), len(pairs)
    s = int(sum(x * (x - 1) * (x - 2) // 6 for x in d))
    p = int(sum((d[a] - 1) * (d[b] - 1) for a, b in pairs))
    return s + p, len(pairs)


def _run(hm, h, k):
    mem = torch.from_numpy(h.members).cuda()
    off = torch.from_numpy(h.offsets).cuda()
    hist, cand, npairs = hm.count_exact_baseline(mem, off, h.num_nodes, k)
    return hist.cpu().numpy().astype(np.uint64), cand, npairs


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("k", [3, 4])
def test_tiny_random(hm, seed, k):
    h = synth.random_tiny(7 + seed % 6, 10 + 3 * seed, max_size=7, seed=200 + seed, dup_frac=0.3)
    got, cand, npairs = _run(hm, h, k)
    want, _ = oracle.Graph.from_hypergraph(h, 4).census(k, threads=os.cpu_count() or 1)
    assert (got == want).all()
    assert (cand, npairs) == _closed_form(h, k)


def test_figure_2_case(hm):
    # one 5-node hyperedge: its projection is K5, so every 3- and 4-set is
    # projection-connected, yet no sub-hypergraph of them has a hyperedge
    h = synth.from_edges([[0, 1, 2, 3, 4]], 6)
    for k in (3, 4):
        got, cand, npairs = _run(hm, h, k)
        assert got.sum() == 0 and npairs == 10
        assert cand == _closed_form(h, k)[0] > 0


@pytest.mark.parametrize("case", ["f2f-330", "coauth-1m-s001"])
@pytest.mark.parametrize("k", [3, 4])
def test_workloads_against_stored_oracle(hm, case, k):
    with open(os.path.join(GOLDEN, f"census_{case}.json")) as f:
        rec = json.load(f)
    h = synth.workload(rec["workload"], seed=rec["seed"], scale=rec["scale"])
    got, cand, npairs = _run(hm, h, k)
    assert got.tolist() == rec["hist"][str(k)]
    assert cand >= int(got.sum())


def test_errors(hm):
    h = synth.from_edges([[0, 9]], 4)
    with pytest.raises(hm.HMError) as e:
        _run(hm, h, 4)
    assert e.value.status == 1
