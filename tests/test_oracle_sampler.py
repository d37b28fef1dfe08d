"""Pins for the oracle's sampling estimator (Alg. 4, Sec. 5), Philox and null model.

* Philox4x32-10 reproduces the published known-answer vectors of Salmon et
  al. (SC'11, Random123 distribution);
* the full-sweep identity: summing the per-hyperedge contributions over all
  hyperedges credits every counted set once per maximum-cardinality
  hyperedge, i.e. countmax_c * T_c (Sec. 5, the max-cardinality rule);
* Alg. 4 run sample by sample equals the same draws summed from the
  contribution table (two independent routes);
* the estimator is unbiased (Sec. 5): the mean over many seeds lies within
  5 standard errors of the exact census, uniform and weighted;
* a constant power-of-two proposal reproduces the uniform estimate exactly;
* the stub shuffle keeps the multiset of stubs and every hyperedge's length.
"""
import numpy as np
import pytest

import oracle
from paper_2209_10241_gb300 import synth


@pytest.mark.parametrize("ctr,key,expected", [
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
])
def test_philox_known_answers(ctr, key, expected):
    assert oracle.philox4x32_10(ctr, key).tolist() == expected


def test_draw64_layout():
    # draw64(seed, index, lane, tag) = (r0 << 32) | r1 of Philox with
    # counter (index lo, index hi, lane, tag) and key (seed lo, seed hi)
    seed, idx, lane, tag = 0x1234_5678_9ABC_DEF0, 0x0000_0007_0000_0003, 4, oracle.TAG_SAMPLE
    r = oracle.philox4x32_10([idx & 0xFFFFFFFF, idx >> 32, lane, tag],
                             [seed & 0xFFFFFFFF, seed >> 32])
    assert oracle.draw64(seed, idx, lane, tag) == (int(r[0]) << 32) | int(r[1])


@pytest.fixture(scope="module")
def small():
    h = synth.workload("uniform-200")
    return h, oracle.Graph.from_hypergraph(h, 4)


def _table_estimate(g, contrib, k, S, seed, q=None):
    """Alg. 4 via the contribution table: sum the rows of the drawn hyperedges."""
    canon, mc, cm = oracle.class_info(k)
    base, off = {}, 0
    for s in range(2, k + 1):
        base[s] = off
        off += g.count(s)
    raw = np.zeros(len(canon), dtype=object)
    for s in range(2, k + 1):
        if g.count(s) == 0 or S[s] == 0:
            continue
        qs = None if q is None else q[base[s]:base[s] + g.count(s)]
        idx = g.sample_indices(s, S[s], seed, qs)
        rows = contrib[base[s] + idx].astype(object)
        if qs is None:
            raw += rows.sum(axis=0)
        else:
            w = np.array([(1 << 63) // int(qs[i]) for i in idx], dtype=object)
            raw += (rows * w[:, None]).sum(axis=0)
    return raw


@pytest.mark.parametrize("k", [3, 4])
def test_full_sweep_identity(small, k):
    h, g = small
    hist, _ = g.census(k, threads=4)
    contrib = g.contributions(k, threads=4)
    _, _, cm = oracle.class_info(k)
    assert (contrib.sum(axis=0).astype(np.uint64) == cm.astype(np.uint64) * hist).all()


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("weighted", [False, True])
def test_direct_equals_table(small, k, weighted):
    h, g = small
    contrib = g.contributions(k, threads=4)
    S = {2: 40, 3: 120, 4: 80}
    q = None
    if weighted:
        rows = contrib.shape[0]
        q = (1 + synth.Stream(5, 9).below(rows, 1000)).astype(np.uint32)
    raw, est, _ = g.sample(k, S, seed=7, q=q)
    table = _table_estimate(g, contrib, k, S, 7, q)
    got = [int(raw[2 * c]) | (int(raw[2 * c + 1]) << 64) for c in range(len(table))]
    assert got == [int(x) for x in table]


def test_power_of_two_proposal_equals_uniform(small):
    h, g = small
    rows = sum(g.count(s) for s in (2, 3, 4))
    S = {2: 50, 3: 150, 4: 100}
    _, est_u, _ = g.sample(4, S, seed=3)
    _, est_w, _ = g.sample(4, S, seed=3, q=np.full(rows, 1 << 12, dtype=np.uint32))
    assert est_u.tobytes() == est_w.tobytes()


def test_uniform_estimate_formula(small):
    h, g = small
    S = {2: 30, 3: 90, 4: 60}
    raw, est, _ = g.sample(4, S, seed=11)
    _, mc, cm = oracle.class_info(4)
    for c in range(len(est)):
        m = int(mc[c])
        want = (float(raw[2 * c]) * float(g.count(m))) / (float(S[m]) * float(cm[c]))
        assert est[c] == want


@pytest.mark.parametrize("weighted", [False, True])
def test_unbiased(small, weighted):
    h, g = small
    k = 3
    hist, _ = g.census(k)
    contrib = g.contributions(k)
    _, mc, cm = oracle.class_info(k)
    S = {2: 25, 3: 75}
    rows = contrib.shape[0]
    q = None
    if weighted:
        # weights loosely following the per-hyperedge totals, floor 1
        q = (1 + contrib.sum(axis=1) // 2).astype(np.uint32)
    R = 400
    ests = []
    for r in range(R):
        raw = _table_estimate(g, contrib, k, S, 1000 + r, q)
        e = []
        for c in range(len(raw)):
            m = int(mc[c])
            Q = g.count(m) if q is None else int(q[(0 if m == 2 else g.count(2)):][:g.count(m)].sum())
            scale = Q / (S[m] * int(cm[c]))
            e.append(float(raw[c]) * scale / (1 if q is None else 2.0 ** 63))
        ests.append(e)
    ests = np.array(ests)
    mean, se = ests.mean(axis=0), ests.std(axis=0, ddof=1) / np.sqrt(R)
    for c in range(len(hist)):
        if hist[c] == 0:
            assert mean[c] == 0
        else:
            assert abs(mean[c] - float(hist[c])) <= 5 * se[c] + 1e-9


def test_stub_shuffle_preserves_stubs_and_sizes():
    h = synth.workload("uniform-200")
    a = oracle.stub_shuffle(h.members, h.offsets, seed=5, model=0)
    b = oracle.stub_shuffle(h.members, h.offsets, seed=5, model=0)
    c = oracle.stub_shuffle(h.members, h.offsets, seed=5, model=1)
    assert (a == b).all() and not (a == c).all()
    assert sorted(a.tolist()) == sorted(h.members.tolist())
    # the permutation is the stable sort of the top 58 bits of the Philox values
    M = h.members.shape[0]
    keys = [(oracle.draw64(5, i, 0, oracle.TAG_NULL) >> 6, i) for i in range(M)]
    order = [i for _, i in sorted(keys)]
    assert a.tolist() == h.members[order].tolist()
