"""GPU parity of Alg. 4 at order 5 (hm_count_sampled5) with the oracle (oracle.sample5).

The GPU enumerates the sets through a draw by ESU from the drawn hyperedge;
the oracle grows every connected superset of it node by node. With the same Philox
draws, the classes met, their raw counts and their estimates must be equal
bit for bit: tiny random hypergraphs with repeated members, duplicates and
hyperedges of 6-7 members, and small face-to-face- and co-authorship-shaped
graphs; plus the default budget split and the errors.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_10241_gb300 import synth

pytestmark = pytest.mark.gpu


def _compare(hm, h, S, seed):
    mem = torch.from_numpy(h.members).cuda()
    off = torch.from_numpy(h.offsets).cuda()
    m, r, e = hm.count_sampled5(mem, off, h.num_nodes, samples=S, seed=seed)
    om, orr, oe = oracle.sample5(h.members, h.offsets, h.num_nodes, S, seed=seed)
    assert np.array_equal(m.cpu().numpy().astype(np.uint32), om)
    assert np.array_equal(r.cpu().numpy().astype(np.uint64), orr)
    assert e.cpu().numpy().tobytes() == oe.tobytes()
    return len(om)


@pytest.mark.parametrize("seed", range(10))
def test_tiny_random(hm, seed):
    h = synth.random_tiny(8 + seed % 4, 16 + 3 * seed, max_size=7, seed=700 + seed,
                          dup_frac=0.2)
    S = {2: 30, 3: 30, 4: 20, 5: 20}
    _compare(hm, h, S, seed=seed)


@pytest.mark.parametrize("name,scale,S", [
    ("f2f-330", 0.05, {2: 20, 3: 40, 4: 30, 5: 20}),
    ("f2f-330", 0.2, {2: 4, 3: 16, 4: 20, 5: 20}),
    ("coauth-1m", 0.005, {2: 100, 3: 100, 4: 100, 5: 100}),
])
def test_workloads(hm, name, scale, S):
    h = synth.workload(name, seed=1, scale=scale)
    assert _compare(hm, h, S, seed=3) > 10


def test_default_split_and_empty_strata(hm):
    h = synth.from_edges([[0, 1], [1, 2], [2, 3], [3, 4], [0, 4], [1, 3]], 6)  # pairs only
    mem = torch.from_numpy(h.members).cuda()
    off = torch.from_numpy(h.offsets).cuda()
    m, r, e = hm.count_sampled5(mem, off, h.num_nodes, total=800, seed=5)
    S = {2: 100, 3: 300, 4: 200, 5: 200}
    om, orr, oe = oracle.sample5(h.members, h.offsets, h.num_nodes, S, seed=5)
    assert np.array_equal(m.cpu().numpy().astype(np.uint32), om)
    assert np.array_equal(r.cpu().numpy().astype(np.uint64), orr)


def test_errors(hm):
    h = synth.from_edges([[0, 1], [1, 2, 3]], 4)
    mem = torch.from_numpy(h.members).cuda()
    off = torch.from_numpy(h.offsets).cuda()
    with pytest.raises(hm.HMError) as e:
        hm.count_sampled5(mem, off, h.num_nodes, samples={2: 5, 3: 0, 4: 0, 5: 0}, seed=1)
    assert e.value.status == 1
