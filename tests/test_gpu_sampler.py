"""GPU parity of the sampling estimator (hm_count_sampled, Alg. 4) against the CPU oracle.

Given the same seed, the draws come from the same Philox stream on both
sides, so the integer accumulators must match bit for bit and the estimates
(evaluated in IEEE double in a fixed order) must be identical.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_10241_gb300 import synth

pytestmark = pytest.mark.gpu


def _compare(hm, h, k, S, seed, q=None, kmax=4):
    g = hm.from_host(h, kmax)
    og = oracle.Graph.from_hypergraph(h, kmax)
    qd = None if q is None else torch.from_numpy(np.asarray(q, dtype=np.int32)).cuda()
    est, raw = hm.count_sampled(g, k, samples=S, seed=seed, q=qd)
    oraw, oest, _ = og.sample(k, S, seed=seed, q=q)
    got_raw = raw.cpu().numpy().astype(np.uint64)
    assert (got_raw == oraw).all(), (got_raw, oraw)
    assert est.cpu().numpy().tobytes() == oest.tobytes()
    return est.cpu().numpy(), got_raw


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [3, 4])
def test_tiny_uniform(hm, seed, k):
    h = synth.random_tiny(9 + seed, 30 + 5 * seed, max_size=5, seed=200 + seed, dup_frac=0.2)
    og = oracle.Graph.from_hypergraph(h, 4)
    S = {s: (7 * s if og.count(s) else 0) for s in range(2, k + 1)}
    _compare(hm, h, k, S, seed=seed)


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("seed", [0, 1, 12345678901234])
def test_uniform_workload(hm, k, seed):
    h = synth.workload("uniform-200")
    S = {2: 500, 3: 1500, 4: 1000}
    _compare(hm, h, k, S, seed=seed)


@pytest.mark.parametrize("k", [3, 4])
def test_weighted_workload(hm, k):
    h = synth.workload("uniform-200")
    og = oracle.Graph.from_hypergraph(h, 4)
    rows = sum(og.count(s) for s in range(2, k + 1))
    q = (1 + synth.Stream(3, 4).below(rows, 5000)).astype(np.uint32)
    S = {2: 400, 3: 1200, 4: 800}
    _compare(hm, h, k, S, seed=9, q=q)


def test_f2f_sampled(hm):
    h = synth.workload("f2f-330")
    S = {2: 60, 3: 180, 4: 120}
    est, _ = _compare(hm, h, 4, S, seed=4)
    assert np.isfinite(est).all()


def test_batches_and_power_of_two_weights(hm):
    # constant power-of-two weights reproduce the uniform estimate exactly
    h = synth.workload("uniform-200")
    g = hm.from_host(h, 4)
    rows = sum(g.count(s) for s in (2, 3, 4))
    S = {2: 3000, 3: 9000, 4: 6000}
    est_u, _ = hm.count_sampled(g, 4, samples=S, seed=5)
    q = torch.full((rows,), 1 << 10, dtype=torch.int32, device="cuda")
    est_w, _ = hm.count_sampled(g, 4, samples=S, seed=5, q=q)
    assert est_u.cpu().numpy().tobytes() == est_w.cpu().numpy().tobytes()


def test_default_split_and_errors(hm):
    h = synth.workload("uniform-200")
    g = hm.from_host(h, 4)
    est_a, raw_a = hm.count_sampled(g, 4, total=6000, seed=2)
    est_b, raw_b = hm.count_sampled(g, 4, samples={2: 1000, 3: 3000, 4: 2000}, seed=2)
    assert torch.equal(raw_a, raw_b)
    with pytest.raises(hm.HMError) as e:
        hm.count_sampled(g, 4, samples={2: 10, 3: 0, 4: 10}, seed=2)
    assert e.value.status == 1
    with pytest.raises(hm.HMError) as e:
        hm.count_sampled(g, 4, samples={2: 10, 3: 10, 4: 10}, seed=2,
                         q=torch.zeros(g.count(2) + g.count(3) + g.count(4), dtype=torch.int32,
                                       device="cuda"))
    assert e.value.status == 1
    # an empty stratum contributes an exact zero
    h2 = synth.from_edges([[0, 1], [1, 2], [2, 3], [0, 1, 2]], 5)
    g2 = hm.from_host(h2, 4)
    est, raw = hm.count_sampled(g2, 4, samples={2: 50, 3: 50, 4: 0}, seed=1)
    og = oracle.Graph.from_hypergraph(h2, 4)
    oraw, oest, _ = og.sample(4, {2: 50, 3: 50, 4: 0}, seed=1)
    assert est.cpu().numpy().tobytes() == oest.tobytes()


def test_trace_filter_keeps_one_kernel(hm):
    g = hm.from_host(synth.workload("uniform-200"), 4)
    hm.trace_read()
    hm.trace_only("census_Q")
    hm.trace_enable(True)
    try:
        hm.count_exact(g, 4)
        torch.cuda.synchronize()
    finally:
        hm.trace_enable(False)
        hm.trace_only(None)
    names = [name for name, _ in hm.trace_read()]
    assert names and set(names) == {"census_Q"}


def test_launch_counter_counts_library_kernels(hm):
    h = synth.workload("uniform-200")
    before = hm.launch_count()
    g = hm.from_host(h, 4)
    hm.count_exact(g, 4)
    # ingest (normalise, sort, CSR, spaces) and census launches: at least 10
    # on any path; the fused small-graph chains keep it near 16
    assert hm.launch_count() - before >= 10


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("weighted", [False, True])
def test_pair_stratum_dense(hm, seed, weighted):
    # many 3- and 4-hyperedges on few nodes: the pair stratum's counts by
    # neighbour type meet every correction (3-hyperedges through both ends of
    # the drawn pair, through one end, 4-hyperedges, sets holding several)
    h = synth.random_tiny(16, 220, max_size=4, seed=300 + seed, dup_frac=0.1)
    og = oracle.Graph.from_hypergraph(h, 4)
    rows = sum(og.count(s) for s in (2, 3, 4))
    q = (1 + synth.Stream(5, seed).below(rows, 1000)).astype(np.uint32) if weighted else None
    _compare(hm, h, 4, {2: 3000, 3: 30, 4: 30}, seed=seed, q=q)


@pytest.mark.parametrize("weighted", [False, True])
def test_pair_stratum_types_equal_enumeration(hm, monkeypatch, weighted):
    # a communication-shaped graph with hubs (5,000 nodes, 10,000 hyperedges):
    # the counts by neighbour type equal the per-candidate enumeration of the
    # pairs' sets (HM_SAMPLE_PAIR_ENUM=1) bit for bit
    h = synth.workload("comm-5m", seed=11, scale=0.001)
    g = hm.from_host(h, 4)
    rows = sum(g.count(s) for s in (2, 3, 4))
    q = None
    if weighted:
        q = torch.from_numpy((1 + synth.Stream(6, 1).below(rows, 1 << 20)).astype(np.int32)).cuda()
    S = {2: 40_000, 3: 10, 4: 10}
    est_t, raw_t = hm.count_sampled(g, 4, samples=S, seed=21, q=q)
    monkeypatch.setenv("HM_SAMPLE_PAIR_ENUM", "1")
    est_e, raw_e = hm.count_sampled(g, 4, samples=S, seed=21, q=q)
    assert torch.equal(raw_t, raw_e)
    assert est_t.cpu().numpy().tobytes() == est_e.cpu().numpy().tobytes()
