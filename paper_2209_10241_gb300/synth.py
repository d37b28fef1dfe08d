"""Seeded synthetic hypergraph generators.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests. It holds no motif-counting arithmetic: it only draws hyperedge lists.

Determinism across machines (x86 here, aarch64 elsewhere, any numpy version):
* randomness comes from a counter-based SplitMix64 stream (Steele, Lea and
  Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
  evaluated with wrapping uint64 numpy arithmetic, so no numpy bit generator
  is involved;
* node weights and size probabilities are quantised to integers before they
  are used, and every draw is an integer inverse-CDF lookup.

The workload shapes stand in for the paper's datasets (Table 1, Sec. 6.1),
which are not available: face-to-face proximity (hs/ps), co-authorship
(dblp/history/geology) and e-mail communication (EU).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise (wrapping uint64)."""
    with np.errstate(over="ignore"):
        z = z.astype(np.uint64, copy=True)
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


class Stream:
    """Counter-based 64-bit random stream: value i = mix64(base + (i+1)*golden)."""

    def __init__(self, seed: int, tag: int = 0):
        s = np.array([(seed * 0x100000001B3 + tag * 0xC2B2AE3D27D4EB4F) & (2**64 - 1)],
                     dtype=np.uint64)
        self._base = _mix64(s)[0]
        self._ctr = 0

    def u64(self, count: int) -> np.ndarray:
        idx = np.arange(self._ctr + 1, self._ctr + 1 + count, dtype=np.uint64)
        self._ctr += count
        with np.errstate(over="ignore"):
            return _mix64(self._base + idx * _GOLDEN)

    def below(self, count: int, bound: int) -> np.ndarray:
        """Integers in [0, bound) (bound < 2**63) by 64-bit modulo reduction."""
        return (self.u64(count) % np.uint64(bound)).astype(np.int64)


def _quantised_cdf(weights: np.ndarray, scale_bits: int) -> np.ndarray:
    w = np.asarray(weights, dtype=np.float64)
    q = np.floor(w / w.max() * float(2**scale_bits) + 0.5).astype(np.int64)
    q = np.maximum(q, 1)
    return np.cumsum(q)


def _draw(cdf: np.ndarray, stream: Stream, count: int) -> np.ndarray:
    r = stream.below(count, int(cdf[-1]))
    return np.searchsorted(cdf, r, side="right").astype(np.int64)


def powerlaw_node_weights(n: int, gamma: float, total_incidences: float) -> np.ndarray:
    """Activity weights w_i = (i + i0)^(-1/(gamma-1)), i = 0..n-1.

    i0 is chosen so that the expected degree of the heaviest node equals
    sqrt(total incidences) (the structural cutoff), then rounded to four
    significant digits so that platform libm differences cannot move it.
    """
    alpha = 1.0 / (gamma - 1.0)
    idx = np.arange(n, dtype=np.float64)
    target = math.sqrt(total_incidences) / total_incidences

    def top_share(i0: float) -> float:
        w = (idx + i0) ** (-alpha)
        return float(w[0] / w.sum())

    lo, hi = 1e-3, 1e12
    if top_share(lo) <= target:
        i0 = lo
    else:
        for _ in range(200):
            mid = math.sqrt(lo * hi)
            if top_share(mid) > target:
                lo = mid
            else:
                hi = mid
        i0 = hi
    i0 = float(f"{i0:.4g}")
    return (idx + i0) ** (-alpha)


@dataclasses.dataclass
class Hypergraph:
    """Flattened hyperedge list: members of hyperedge j are members[offsets[j]:offsets[j+1]]."""
    members: np.ndarray   # int32
    offsets: np.ndarray   # int64, len m+1
    num_nodes: int
    name: str = ""

    @property
    def num_hyperedges(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def edges(self):
        m, o = self.members, self.offsets
        return [m[o[j]:o[j + 1]].tolist() for j in range(self.num_hyperedges)]


def from_edges(edges, num_nodes: int, name: str = "") -> Hypergraph:
    sizes = np.array([len(e) for e in edges], dtype=np.int64)
    offsets = np.zeros(len(edges) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    members = (np.concatenate([np.asarray(e, dtype=np.int32) for e in edges])
               if len(edges) and offsets[-1] > 0 else np.zeros(0, dtype=np.int32))
    return Hypergraph(members.astype(np.int32), offsets, int(num_nodes), name)


def generate(n: int, m: int, size_values, size_probs, gamma=None, seed: int = 0,
             shuffle_ids: bool = True, name: str = "", batch: int = 1 << 21) -> Hypergraph:
    """Draw m distinct hyperedges.

    Sizes are drawn from (size_values, size_probs); members are drawn i.i.d.
    from the node weights (uniform when gamma is None) and a candidate with a
    repeated member is redrawn (conditional sampling without replacement).
    Duplicate hyperedges are rejected (E is a set, Def. 1) until m distinct
    ones exist; the output keeps draw order and the drawn member order. Node
    ids are finally relabelled by a seeded permutation, so that hubs do not
    sit at the smallest ids.
    """
    size_values = np.asarray(size_values, dtype=np.int64)
    size_cdf = _quantised_cdf(np.asarray(size_probs, dtype=np.float64), 32)
    mean_size = float(np.dot(size_values, np.asarray(size_probs)) / np.sum(size_probs))
    if gamma is None:
        node_cdf = np.arange(1, n + 1, dtype=np.int64)
    else:
        node_cdf = _quantised_cdf(powerlaw_node_weights(n, gamma, m * mean_size), 36)
    width = int(size_values.max())
    st_size = Stream(seed, 1)
    st_node = Stream(seed, 2)
    st_perm = Stream(seed, 3)

    kept_sorted = np.zeros((0, width), dtype=np.int32)
    kept_raw = np.zeros((0, width), dtype=np.int32)
    kept_size = np.zeros(0, dtype=np.int64)
    while kept_sorted.shape[0] < m:
        need = m - kept_sorted.shape[0]
        b = int(min(batch, max(1024, need * 1.25 + 64)))
        sizes = size_values[np.searchsorted(size_cdf, st_size.below(b, int(size_cdf[-1])),
                                            side="right")]
        raw = _draw(node_cdf, st_node, b * width).reshape(b, width).astype(np.int32)
        col = np.arange(width)[None, :]
        valid = col < sizes[:, None]
        raw = np.where(valid, raw, n).astype(np.int32)
        srt = np.sort(raw, axis=1)
        rep = np.any((srt[:, 1:] == srt[:, :-1]) & (srt[:, 1:] < n), axis=1)
        keep = ~rep
        srt, raw, sizes = srt[keep], raw[keep], sizes[keep]
        all_sorted = np.concatenate([kept_sorted, srt])
        all_raw = np.concatenate([kept_raw, raw])
        all_size = np.concatenate([kept_size, sizes])
        _, first = np.unique(all_sorted, axis=0, return_index=True)
        first = np.sort(first)[:m]
        kept_sorted, kept_raw, kept_size = all_sorted[first], all_raw[first], all_size[first]

    perm = np.argsort(st_perm.u64(n), kind="stable").astype(np.int32)
    perm_ext = np.concatenate([perm, np.array([n], dtype=np.int32)])
    relabelled = perm_ext[kept_raw] if shuffle_ids else kept_raw
    col = np.arange(width)[None, :]
    members = relabelled[col < kept_size[:, None]]
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(kept_size, out=offsets[1:])
    return Hypergraph(members.astype(np.int32), offsets, n, name)


def _trunc_powerlaw(lo: int, hi: int, exponent: float):
    s = np.arange(lo, hi + 1)
    return s, s.astype(np.float64) ** (-exponent)


def _geometric(lo: int, hi: int, ratio: float):
    s = np.arange(lo, hi + 1)
    return s, ratio ** (s - 1).astype(np.float64)


# Workloads. Sizes stand in for the paper's datasets (Table 1, Sec. 6.1).
WORKLOADS = {
    # small exact order-3 (and order-4) census case
    "uniform-200": dict(n=200, m=2000, sizes=([2, 3, 4], [0.6, 0.3, 0.1]), gamma=None),
    # face-to-face proximity shaped (hs / ps)
    "f2f-330": dict(n=330, m=20000, sizes=([2, 3, 4, 5], [0.70, 0.22, 0.06, 0.02]), gamma=2.5),
    # co-authorship shaped (dblp / history / geology)
    "coauth-1m": dict(n=1_000_000, m=2_000_000, sizes=_trunc_powerlaw(2, 25, 2.5), gamma=2.2),
    # e-mail communication shaped (EU)
    "comm-5m": dict(n=5_000_000, m=10_000_000, sizes=_geometric(2, 10, 0.5), gamma=2.0),
}


def workload(name: str, seed: int = 0, scale: float = 1.0) -> Hypergraph:
    """Generate a named workload; scale multiplies both n and m (for smaller stand-ins)."""
    w = WORKLOADS[name]
    n = max(8, int(round(w["n"] * scale)))
    m = max(4, int(round(w["m"] * scale)))
    return generate(n, m, w["sizes"][0], w["sizes"][1], w["gamma"], seed=seed, name=name)


def null_base(hyperedges: int, seed: int) -> Hypergraph:
    """Face-to-face shaped base graph for the null-model batch, at constant density.

    330 nodes cannot hold 500k distinct hyperedges of that size mix, so the node
    count grows with the hyperedge count: n = 330 * H / 20000.
    """
    w = WORKLOADS["f2f-330"]
    n = max(16, int(round(330 * hyperedges / 20000)))
    return generate(n, hyperedges, w["sizes"][0], w["sizes"][1], w["gamma"], seed=seed,
                    name=f"f2f-null-{hyperedges}")


def random_tiny(n: int, m: int, max_size: int, seed: int, dup_frac: float = 0.0) -> Hypergraph:
    """Small random hypergraph with raw (possibly repeated, unsorted) members.

    Sizes are uniform in [1, max_size]; with dup_frac > 0 some hyperedges are
    repeated with shuffled member order and repeated members, to exercise
    normalisation.
    """
    st = Stream(seed, 7)
    edges = []
    for _ in range(m):
        s = 1 + int(st.below(1, max_size)[0])
        edges.append([int(x) for x in st.below(s, n)])
    extra = int(m * dup_frac)
    for j in range(extra):
        src = edges[int(st.below(1, len(edges))[0])]
        rot = int(st.below(1, max(1, len(src)))[0])
        e = src[rot:] + src[:rot]
        if e:
            e = e + [e[0]]
        edges.append(e)
    return from_edges(edges, n, name=f"tiny-{n}-{m}-{seed}")


def mlp_init_params(seed: int) -> np.ndarray:
    """Seeded He-uniform initial weights of the 16-64-64-1 proposal MLP
    (packed W1[16][64] | b1 | W2[64][64] | b2 | w3[64] | b3, float32)."""
    n_in, hid = 16, 64
    sizes = [n_in * hid, hid, hid * hid, hid, hid, 1]
    total = sum(sizes)
    st = Stream(seed, 11)
    u = (st.u64(total) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    p = np.zeros(total)
    o_w1, o_w2 = 0, n_in * hid + hid
    o_w3 = o_w2 + hid * hid + hid
    p[o_w1:o_w1 + n_in * hid] = (2 * u[o_w1:o_w1 + n_in * hid] - 1) * np.sqrt(6.0 / n_in)
    p[o_w2:o_w2 + hid * hid] = (2 * u[o_w2:o_w2 + hid * hid] - 1) * np.sqrt(6.0 / hid)
    p[o_w3:o_w3 + hid] = (2 * u[o_w3:o_w3 + hid] - 1) * np.sqrt(6.0 / hid)
    return p.astype(np.float32)
