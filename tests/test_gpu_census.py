"""GPU parity of the exact census (hm_build + hm_count_exact) against the CPU oracle.

Counts are integers and must match bit for bit. Cases span tiny hypergraphs
with every normalisation edge case, closed-form families, the workloads at
their full sizes (stored oracle histograms), every candidate-evaluation path
(pair probes in the hash set or the dense bitmap, per-candidate or
bit-sliced families) and the error paths of the C ABI.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2209_10241_gb300 import synth
from tests.golden.make_golden import input_digest

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


MODES = ["hash", "bitmap", "sliced", "sliced_filter", "tuned", "chunk8", "chunk32", "graphlets",
         "graphlets_filter", "graphlets_pc", "graphlets_hash", "graphlets_tiers",
         "graphlets_sort"]


def _set_mode(monkeypatch, mode):
    """hash: pair probes in the hash set; bitmap: pair probes in the dense
    bitmap, one candidate at a time; sliced: bit-sliced W/S/P families with
    exact 3-hyperedge rows; sliced_filter: bit-sliced with the co-occurrence
    filter and exact probes of the risky candidates; tuned: the library's
    defaults, schedules picked by the autotuner; chunk8 / chunk32: hash
    probes with 8 / 32 candidates per lane on every per-candidate family
    (chunk8 with TX per candidate too, else TX goes by 3-hyperedge with node
    signatures); graphlets*: pairs-only sets from graphlet identities, with the bit-sliced
    TX family on exact rows / on the co-occurrence filter (and a warp per
    pair on short rows) / per candidate;
    graphlets_hash: the same without pair bitmaps (hash probes, 4-cycles by
    degree order); graphlets_tiers: graphlets_hash with the warp tier of the
    4-cycle pass bounded at 4 paths, so that small graphs' nodes reach the
    per-node table tier too, and the per-node sums taken over the whole
    grid; graphlets_sort: graphlets_tiers with the heavy nodes' 4-cycles
    counted by sorting their path keys instead of per-node tables."""
    for var in ("HM_PAIR_BITMAP", "HM_DENSE_FAMILIES", "HM_TRIPLE_ROWS", "HM_AUTOTUNE",
                "HM_CENSUS_CHUNK", "HM_GRAPHLETS", "HM_C4_UB", "HM_GL_NODE_SUMS", "HM_GL_WIDE",
                "HM_TX_PER_CANDIDATE", "HM_C4_SORT"):
        monkeypatch.delenv(var, raising=False)
    if mode == "tuned":
        return
    if mode in ("graphlets_hash", "graphlets_tiers", "graphlets_sort"):
        monkeypatch.setenv("HM_PAIR_BITMAP", "0")
        monkeypatch.setenv("HM_GRAPHLETS", "1")
        monkeypatch.setenv("HM_AUTOTUNE", "0")
        if mode != "graphlets_hash":
            monkeypatch.setenv("HM_C4_UB", "4")
            monkeypatch.setenv("HM_GL_NODE_SUMS", "1")
        if mode == "graphlets_sort":
            monkeypatch.setenv("HM_C4_SORT", "1")
        return
    if mode.startswith("graphlets"):
        monkeypatch.setenv("HM_PAIR_BITMAP", "1")
        monkeypatch.setenv("HM_GRAPHLETS", "1")
        monkeypatch.setenv("HM_AUTOTUNE", "0")
        monkeypatch.setenv("HM_TRIPLE_ROWS", "0" if mode == "graphlets_filter" else "1")
        if mode == "graphlets_filter":
            monkeypatch.setenv("HM_GL_WIDE", "1")
        monkeypatch.setenv("HM_DENSE_FAMILIES", "0" if mode == "graphlets_pc" else "1")
        return
    if mode.startswith("chunk"):
        monkeypatch.setenv("HM_PAIR_BITMAP", "0")
        monkeypatch.setenv("HM_CENSUS_CHUNK", mode[5:])
        if mode == "chunk8":
            monkeypatch.setenv("HM_TX_PER_CANDIDATE", "1")
        return
    monkeypatch.setenv("HM_PAIR_BITMAP", "0" if mode == "hash" else "1")
    monkeypatch.setenv("HM_DENSE_FAMILIES", "1" if mode.startswith("sliced") else "0")
    monkeypatch.setenv("HM_TRIPLE_ROWS", "0" if mode == "sliced_filter" else "1")


@pytest.fixture(params=MODES)
def pair_path(request, monkeypatch):
    _set_mode(monkeypatch, request.param)
    return request.param


def _gpu_hist(hm, h, k, kmax=4):
    g = hm.from_host(h, kmax)
    out = hm.count_exact(g, k).cpu().numpy().astype(np.uint64)
    return out, g


def _oracle_hist(h, k, kmax=4):
    return oracle.Graph.from_hypergraph(h, kmax).census(k, threads=os.cpu_count() or 1)[0]


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("k", [3, 4])
def test_tiny_random(hm, pair_path, seed, k):
    n = 6 + seed % 5
    h = synth.random_tiny(n, 8 + 3 * seed, max_size=6, seed=seed, dup_frac=0.3)
    got, g = _gpu_hist(hm, h, k)
    want = _oracle_hist(h, k)
    assert (got == want).all(), (got, want)


@pytest.mark.parametrize("seed", range(4))
def test_denser_random(hm, pair_path, seed):
    # many overlapping hyperedges on few nodes: every family and rule fires
    h = synth.random_tiny(14, 160, max_size=4, seed=100 + seed, dup_frac=0.1)
    for k in (3, 4):
        got, _ = _gpu_hist(hm, h, k)
        assert (got == _oracle_hist(h, k)).all()


def test_normalised_hyperedges_match_oracle(hm):
    h = synth.random_tiny(40, 600, max_size=6, seed=5, dup_frac=0.5)
    g = hm.from_host(h, 4)
    og = oracle.Graph.from_hypergraph(h, 4)
    for s in (2, 3, 4):
        assert g.count(s) == og.count(s)
        assert (g.edges(s).cpu().numpy() == og.edges(s)).all()
    assert g.counts[5] == og.count(5)


@pytest.mark.parametrize("name", ["K7", "star9", "path12", "cycle13", "tri6", "mixed"])
def test_closed_forms(hm, pair_path, name):
    n = 14
    edges = {
        "K7": [[a, b] for a in range(7) for b in range(a + 1, 7)],
        "star9": [[0, i] for i in range(1, 10)],
        "path12": [[i, i + 1] for i in range(11)],
        "cycle13": [[i, (i + 1) % 13] for i in range(13)],
        "tri6": [[a, b, c] for a in range(6) for b in range(a + 1, 6) for c in range(b + 1, 6)],
        "mixed": [[0, 1, 2, 3], [0, 1, 2], [1, 2], [2, 3], [3, 4], [4, 5, 6], [0, 1, 2, 3, 4]],
    }[name]
    h = synth.from_edges(edges, n)
    for k in (3, 4):
        got, _ = _gpu_hist(hm, h, k)
        assert (got == _oracle_hist(h, k)).all()


def _golden(case):
    with open(os.path.join(GOLDEN, f"census_{case}.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("case", ["uniform-200", "f2f-330", "coauth-1m-s001"])
@pytest.mark.parametrize("k", [3, 4])
def test_workloads_against_stored_oracle(hm, case, k):
    rec = _golden(case)
    h = synth.workload(rec["workload"], seed=rec["seed"], scale=rec["scale"])
    assert input_digest(h) == rec["input_sha256"], "generator drift: regenerate goldens"
    got, g = _gpu_hist(hm, h, k)
    for s in (2, 3, 4):
        assert g.count(s) == rec["distinct_per_size"][str(s)]
    assert got.tolist() == rec["hist"][str(k)]


@pytest.mark.parametrize("case", ["f2f-330", "coauth-1m-s001"])
@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("mode", MODES)
def test_workload_every_path(hm, monkeypatch, case, k, mode):
    _set_mode(monkeypatch, mode)
    rec = _golden(case)
    h = synth.workload(rec["workload"], seed=rec["seed"], scale=rec["scale"])
    got, _ = _gpu_hist(hm, h, k)
    assert got.tolist() == rec["hist"][str(k)]


@pytest.mark.parametrize("count", [1, 1023, 1024, 1025, 2049, 5000, 8192, 8193, 20000])
@pytest.mark.parametrize("bitmap", ["0", "1"])
def test_ingest_sort_sizes(hm, monkeypatch, count, bitmap):
    # exactly `count` 3- and 4-hyperedges each (a fifth of them repeats): the
    # one-block sort (1..8 keys per thread, <= 8192 keys) and the multi-tile
    # sort, each side of every threshold, with and without pair bitmaps
    monkeypatch.setenv("HM_PAIR_BITMAP", bitmap)
    n = 300
    st = synth.Stream(11, count)
    edges = []
    for size in (3, 4):
        u = st.u64(2 * count * size).reshape(2 * count, size)
        rows = [sorted(set(int(x) for x in r)) for r in (u % n)]
        rows = [r for r in rows if len(r) == size]
        base = count - count // 5
        rows = rows[:base] + rows[: count - base]
        assert len(rows) == count
        edges += rows
    h = synth.from_edges(edges, n)
    g = hm.from_host(h, 4)
    og = oracle.Graph.from_hypergraph(h, 4)
    for s in (2, 3, 4):
        assert g.count(s) == og.count(s)
        assert (g.edges(s).cpu().numpy() == og.edges(s)).all()


@pytest.mark.parametrize("bitmap", ["0", "1"])
@pytest.mark.parametrize("m", [1, 31, 1023, 1024, 3001])
def test_normalise_long_member_lists(hm, monkeypatch, bitmap, m):
    # hyperedges of 2-6 members, every 13th one a long list (up to 400
    # entries, most of them repeats of at most five distinct members, or a
    # set of 60 distinct members): a warp's member range then exceeds what it
    # stages in shared memory and the rest is read directly; m not a
    # multiple of the per-block tile (ragged last block)
    monkeypatch.setenv("HM_PAIR_BITMAP", bitmap)
    n = 500
    st = synth.Stream(29, m)
    u = st.u64(8 * m).reshape(m, 8)
    edges = []
    for j in range(m):
        r = u[j]
        if j % 13 == 5:
            base = [int(x % n) for x in r[:2 + int(r[7] % 4)]]
            edges.append(base * (400 // len(base)))
        elif j % 13 == 9:
            edges.append([(int(r[0]) + 7 * i) % n for i in range(60)])
        else:
            edges.append([int(x % n) for x in r[:2 + int(r[6] % 5)]])
    h = synth.from_edges(edges, n)
    g = hm.from_host(h, 4)
    og = oracle.Graph.from_hypergraph(h, 4)
    for s in (2, 3, 4):
        assert g.count(s) == og.count(s)
        assert (g.edges(s).cpu().numpy() == og.edges(s)).all()
    assert g.counts[5] == og.count(5)


def test_relabel_and_duplicate_invariance(hm, pair_path):
    h = synth.workload("uniform-200")
    base = {k: _gpu_hist(hm, h, k)[0] for k in (3, 4)}
    st = synth.Stream(7, 1)
    perm = np.argsort(st.u64(h.num_nodes), kind="stable").astype(np.int32)
    edges = [list(perm[np.asarray(e)]) for e in h.edges()]
    edges = edges[::-1] + edges[:500] + [[e[0]] for e in edges[:50]]
    h2 = synth.from_edges(edges, h.num_nodes)
    for k in (3, 4):
        assert (_gpu_hist(hm, h2, k)[0] == base[k]).all()


def test_repeated_counts_are_identical(hm):
    h = synth.workload("uniform-200")
    g = hm.from_host(h, 4)
    a = hm.count_exact(g, 4).cpu()
    b = hm.count_exact(g, 4).cpu()
    assert torch.equal(a, b)


def test_empty_and_degenerate_inputs(hm, pair_path):
    # no hyperedges
    h = synth.from_edges([], 5)
    for k in (3, 4):
        assert _gpu_hist(hm, h, k)[0].sum() == 0
    # singletons, repeated members only, oversized hyperedges only
    h = synth.from_edges([[1], [2, 2, 2], [0, 1, 2, 3, 4]], 6)
    g = hm.from_host(h, 4)
    assert [g.count(s) for s in (2, 3, 4)] == [0, 0, 0] and g.counts[5] == 1
    assert hm.count_exact(g, 4).sum().item() == 0
    # a single node
    h = synth.from_edges([[0, 0]], 1)
    assert _gpu_hist(hm, h, 3)[0].sum() == 0


def test_abi_errors(hm):
    h = synth.from_edges([[0, 1], [1, 7]], 5)   # member 7 outside [0, 5)
    with pytest.raises(hm.HMError) as e:
        hm.from_host(h, 4)
    assert e.value.status == 1
    # an out-of-range member after the fifth distinct one (past where the
    # normalisation stops reading a hyperedge) and a negative one
    for bad in (9, -1):
        h = synth.from_edges([[0, 1], [0, 1, 2, 3, 4, 5, bad]], 8)
        with pytest.raises(hm.HMError) as e:
            hm.from_host(h, 4)
        assert e.value.status == 1
    g = hm.from_host(synth.from_edges([[0, 1], [1, 2]], 3), 3)
    with pytest.raises(hm.HMError) as e:
        hm.count_exact(g, 4)
    assert e.value.status == 6
    with pytest.raises(hm.HMError) as e:
        hm.count_exact(g, 5)
    assert e.value.status == 1
    assert hm.num_classes(3) == 6 and hm.num_classes(4) == 171 and hm.num_classes(5) == -1


def test_l2_read_bandwidth_probe(hm):
    # instrumentation for the L2 roofline: a finite positive rate, and
    # sizes outside (0, 64 MiB] or not a multiple of 16 rejected
    bw = hm.l2_read_bandwidth(16 << 20, 4)
    assert np.isfinite(bw) and bw > 0
    for bad in (0, 100, (64 << 20) + 16):
        with pytest.raises(hm.HMError) as e:
            hm.l2_read_bandwidth(bad, 1)
        assert e.value.status == 1


@pytest.mark.parametrize("k", [3, 4])
def test_class_table_matches_oracle(hm, k):
    canon, mc, cm = oracle.class_info(k)
    for c in range(len(canon)):
        assert hm.class_info(k, c) == (int(canon[c]), int(mc[c]), int(cm[c]))
    for mask in range(1 << (4 if k == 3 else 11)):
        assert hm.class_of_mask(k, mask) == oracle.class_of(k, mask)


def test_full_size_coauthorship_paths_agree(hm, monkeypatch):
    # at full size (10^6 nodes, 2.10^6 hyperedges) the oracle is too slow for
    # the whole census, so two independent GPU paths must agree bit for bit:
    # the graphlet identities with hash probes against the per-candidate S/P
    # enumeration (each on its own graph build)
    h = synth.workload("coauth-1m")
    hists = []
    for graphlets in ("1", "0"):
        for var in ("HM_PAIR_BITMAP", "HM_DENSE_FAMILIES", "HM_TRIPLE_ROWS", "HM_CENSUS_CHUNK",
                    "HM_C4_UB", "HM_GL_NODE_SUMS", "HM_GL_WIDE", "HM_TX_PER_CANDIDATE",
                    "HM_C4_SORT"):
            monkeypatch.delenv(var, raising=False)
        monkeypatch.setenv("HM_GRAPHLETS", graphlets)
        monkeypatch.setenv("HM_AUTOTUNE", "0")
        g = hm.from_host(h, 4)
        hists.append(hm.count_exact(g, 4).cpu().numpy().astype(np.uint64))
        g.free()
    assert hists[0].sum() > 0
    assert (hists[0] == hists[1]).all()
