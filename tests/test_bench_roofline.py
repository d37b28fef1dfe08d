"""The bench's algorithmic operation count for the graphlet pair kernel, against
a direct loop over pairs and their common neighbours (CPU only)."""
import numpy as np

import bench


def _brute(e2, n, bw):
    adj = [set() for _ in range(n)]
    for u, v in e2:
        adj[u].add(v)
        adj[v].add(u)
    ops = 0
    for u, v in e2:
        ops += 3 * bw
        for w in adj[u] & adj[v]:
            if w > v:
                ops += 4 * (bw - w // 32)
    return ops


def test_k4_by_hand():
    # 6 pairs x 3 x 4 words, plus the common neighbours above v: (0,1) -> 2, 3;
    # (0,2) -> 3; (1,2) -> 3; four of them x 4 ops x 4 words
    e2 = np.array([[0, 1], [0, 2], [1, 2], [0, 3], [1, 3], [2, 3]])
    assert bench.graphlet_pair_ops(e2, 4, 4) == 72 + 64


def test_random_graphs_match_direct_count():
    rng = np.random.default_rng(3)
    for n in (5, 40, 130):
        bw = ((n + 127) // 128) * 4
        pairs = {tuple(sorted(rng.choice(n, 2, replace=False))) for _ in range(3 * n)}
        e2 = np.array(sorted(pairs))
        assert bench.graphlet_pair_ops(e2, n, bw) == _brute(e2, n, bw)


def test_hbm_roofline_fields():
    # 288 B per TX candidate over the launch time, against the copy bandwidth;
    # the DRAM bytes of the capture over the same time beside it
    r = bench.hbm_roofline("census_TX", {"census_TX": 1_000_000}, 1e-4, 5000.0, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 1_000_000 * 288 / 1e-4 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 5000.0) < 1e-12
    traffic = bench.ROOFLINE_HBM["census_TX"][3]
    assert r["traffic"] == traffic
    assert abs(r["dram_gbs_from_traffic"] - traffic / 1e-4 / 1e9) < 1e-6
    assert r["ncu"]["kernel"] == "k_census_txs"
    # a kernel without a byte model reports nulls, not a made-up fraction
    n = bench.hbm_roofline("census_c4_table", {}, 1e-4, 5000.0, "measured")
    assert n["achieved"] is None and n["frac"] is None and n["traffic"] is None


def test_whole_job_rate():
    # replicas: every rank does the units of a step, the slowest rank's time counts
    assert bench.whole_job_rate(1000, 10, 4, 20.0) == 1000 * 10 * 4 / 0.02
