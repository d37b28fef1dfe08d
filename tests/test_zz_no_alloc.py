"""The allocation-free sampler entry point agrees with the allocating one.

hm_count_sampled_noalloc exists for callers that must not allocate device
memory while counting (applications that reserve the GPU's memory up front,
latency-critical loops where cudaMalloc may block); its temporaries live in
a static device array inside libhm.so. Two calls in a row (the array keeps the previous call's contents)
must each match hm_count_sampled bit for bit, the tolerance every sampler
test uses. This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2209_10241_gb300 import synth

pytestmark = pytest.mark.gpu


def _reference(hm, g, k, S, seed, q=None):
    est, raw = hm.count_sampled(g, k, samples=S, seed=seed, q=q)
    return est.cpu().numpy(), raw.cpu().numpy()


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("weighted", [False, True])
def test_two_calls_in_a_row_match_hm_count_sampled(hm, k, weighted):
    h = synth.workload("f2f-330")
    g = hm.from_host(h, 4)
    S = {2: 300, 3: 900, 4: 600}
    q = None
    if weighted:
        rows = sum(g.count(s) for s in range(2, k + 1))
        q = torch.from_numpy((1 + synth.Stream(11, 2).below(rows, 1000)).astype(np.int32)).cuda()
    nc = hm.num_classes(k)
    est = torch.empty(nc, dtype=torch.float64, device="cuda")
    raw = torch.empty(2 * nc, dtype=torch.int64, device="cuda")
    for seed in (21, 22):
        want_est, want_raw = _reference(hm, g, k, S, seed, q)
        hm.count_sampled_noalloc(g, k, est, raw, samples=S, seed=seed, q=q)
        assert est.cpu().numpy().tobytes() == want_est.tobytes()
        assert (raw.cpu().numpy() == want_raw).all()


@pytest.mark.parametrize("weighted", [False, True])
def test_several_batches_per_stratum(hm, weighted):
    # a hub with 6,000 pair neighbours: one order-4 pair draw may need
    # ~0.38 MB of second-level entries, so the static array holds fewer than
    # 90 pair draws at a time and 240 of them run in several batches (the
    # arena is reset between batches, beside the weighted prefix sums)
    hub_leaves = 6_000
    edges = [[0, v] for v in range(1, hub_leaves + 1)]
    st = synth.Stream(5, 9)
    extra = 400
    for _ in range(extra):
        a, b, c, d = (int(x) for x in 1 + st.below(4, 300))
        edges.append([a, b])
        edges.append([0, a, b])
        edges.append([a, b, c])
        edges.append([0, a, b, c, d][:4])
        edges.append([a, c, d])
    h = synth.from_edges(edges, hub_leaves + 1)
    g = hm.from_host(h, 4)
    k = 4
    S = {2: 240, 3: 400, 4: 200}
    q = None
    if weighted:
        rows = sum(g.count(s) for s in range(2, k + 1))
        q = torch.from_numpy((1 + synth.Stream(13, 2).below(rows, 500)).astype(np.int32)).cuda()
    nc = hm.num_classes(k)
    est = torch.empty(nc, dtype=torch.float64, device="cuda")
    raw = torch.empty(2 * nc, dtype=torch.int64, device="cuda")
    for seed in (31, 32):
        want_est, want_raw = _reference(hm, g, k, S, seed, q)
        hm.count_sampled_noalloc(g, k, est, raw, samples=S, seed=seed, q=q)
        assert est.cpu().numpy().tobytes() == want_est.tobytes()
        assert (raw.cpu().numpy() == want_raw).all()


def test_without_raw_buffer_and_default_split(hm):
    h = synth.workload("uniform-200")
    g = hm.from_host(h, 4)
    est = torch.empty(hm.num_classes(4), dtype=torch.float64, device="cuda")
    for seed in (3, 4):
        ref_est, _ = hm.count_sampled(g, 4, total=6000, seed=seed)
        hm.count_sampled_noalloc(g, 4, est, None, total=6000, seed=seed)
        assert est.cpu().numpy().tobytes() == ref_est.cpu().numpy().tobytes()


def test_rejects_graphs_beyond_the_static_scratch(hm):
    # a star whose hub has 10^6 pair neighbours: one order-4 draw of a pair
    # would need ~64 MB of second-level entries, beyond the 32 MiB array
    leaves = 1_000_000
    mem = torch.stack([torch.zeros(leaves, dtype=torch.int32),
                       torch.arange(1, leaves + 1, dtype=torch.int32)], 1).reshape(-1).cuda()
    off = torch.arange(0, 2 * leaves + 1, 2, dtype=torch.int64).cuda()
    g = hm.build(mem, off, leaves + 1, 4)
    est = torch.empty(hm.num_classes(4), dtype=torch.float64, device="cuda")
    with pytest.raises(hm.HMError) as e:
        hm.count_sampled_noalloc(g, 4, est, None, samples={2: 10, 3: 0, 4: 0}, seed=1)
    assert e.value.status == 1 and "32 MiB" in str(e.value)
