"""GPU parity of the null-model batch (hm_count_null_batch) against the CPU oracle.

Each model is the oracle's stub shuffle of its base with the same Philox
stream, normalised and counted by the oracle's exact census; every histogram
row must match bit for bit, for unions of uneven models, more than 64
models (several unions), and every candidate-evaluation path.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2209_10241_gb300 import synth

pytestmark = pytest.mark.gpu


def _oracle_rows(bases, k, J, seed):
    rows = []
    for b, h in enumerate(bases):
        for j in range(J):
            t = b * J + j
            mem = oracle.stub_shuffle(h.members, h.offsets, seed=seed, model=t)
            g = oracle.Graph(mem, h.offsets, h.num_nodes, 4)
            rows.append(g.census(k, threads=os.cpu_count() or 1)[0])
    return np.array(rows, dtype=np.uint64)


@pytest.mark.parametrize("mode", ["hash", "bitmap", "sliced"])
@pytest.mark.parametrize("k", [3, 4])
def test_uneven_models(hm, monkeypatch, mode, k):
    monkeypatch.setenv("HM_PAIR_BITMAP", "0" if mode == "hash" else "1")
    monkeypatch.setenv("HM_DENSE_FAMILIES", "1" if mode == "sliced" else "0")
    monkeypatch.setenv("HM_TRIPLE_ROWS", "1")  # unions never use them: still the filter path
    bases = [synth.workload("f2f-330", seed=1, scale=0.05),
             synth.random_tiny(25, 120, max_size=5, seed=3),
             synth.workload("uniform-200", seed=2, scale=0.3)]
    J = 3
    got = hm.null_batch(bases, k, J, seed=77).cpu().numpy().astype(np.uint64)
    want = _oracle_rows(bases, k, J, seed=77)
    assert got.shape == want.shape
    assert (got == want).all()


def test_more_than_64_models(hm):
    bases = [synth.random_tiny(12, 40, max_size=4, seed=8),
             synth.random_tiny(18, 60, max_size=4, seed=9)]
    J = 35
    got = hm.null_batch(bases, 4, J, seed=5).cpu().numpy().astype(np.uint64)
    want = _oracle_rows(bases, 4, J, seed=5)
    assert (got == want).all()


def test_rows_equal_single_graph_counts(hm):
    import torch
    h = synth.workload("uniform-200", seed=4, scale=0.5)
    J = 4
    rows = hm.null_batch([h], 4, J, seed=11).cpu()
    for t in range(J):
        mem = oracle.stub_shuffle(h.members, h.offsets, seed=11, model=t)
        g = hm.build(torch.from_numpy(mem).cuda(), torch.from_numpy(h.offsets).cuda(),
                     h.num_nodes, 4)
        assert torch.equal(hm.count_exact(g, 4).cpu(), rows[t])


def test_null_batch_errors(hm):
    h = synth.from_edges([[0, 1], [1, 9]], 5)  # member 9 outside [0, 5)
    with pytest.raises(hm.HMError) as e:
        hm.null_batch([h], 4, 2, seed=1)
    assert e.value.status == 1
