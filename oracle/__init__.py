"""CPU oracle for higher-order motif counting (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
may import this package. The CUDA path never does, and the oracle never
imports the CUDA path. See ``oracle.cpp`` for what each function computes and
which passage of the paper it follows.

Parity of the MLP reference (``mlp.py``) and of the feature definition
(``features.py``) is pinned by finite differences and by closed forms in the
tests; the Philox generator is pinned by the published known-answer vectors.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

TAG_SAMPLE = 0x53414D50
TAG_NULL = 0x4E554C4C


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (plain g++, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
               _SRC, "-o", _LIB + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        u64, i64, i32, u32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        vp = ctypes.c_void_p
        sig = {
            "orc_philox4x32_10": (None, [vp, vp, vp]),
            "orc_draw64": (u64, [u64, u64, u32, u32]),
            "orc_num_classes": (ctypes.c_int, [ctypes.c_int]),
            "orc_class_info": (None, [ctypes.c_int, vp, vp, vp]),
            "orc_class_of": (ctypes.c_int, [ctypes.c_int, u32]),
            "orc_canonical": (u32, [ctypes.c_int, u32]),
            "orc_connected": (ctypes.c_int, [ctypes.c_int, u32]),
            "orc_graph_new": (vp, [vp, vp, i64, i32, ctypes.c_int]),
            "orc_graph_free": (None, [vp]),
            "orc_graph_count": (i64, [vp, ctypes.c_int]),
            "orc_graph_edges": (None, [vp, ctypes.c_int, vp]),
            "orc_fill_in": (u32, [vp, ctypes.c_int, vp]),
            "orc_census": (i64, [vp, ctypes.c_int, ctypes.c_int, i64, i64, vp]),
            "orc_contributions": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp]),
            "orc_sample_indices": (None, [vp, ctypes.c_int, u64, u64, vp, vp]),
            "orc_sample": (i64, [vp, ctypes.c_int, vp, u64, vp, vp, vp]),
            "orc_stub_shuffle": (None, [vp, vp, i64, u64, u32, vp]),
            "orc_config_mcmc": (None, [vp, vp, i64, u64, u32, ctypes.c_int, vp]),
            "orc_sample5": (i64, [vp, vp, i64, i32, vp, u64, i64, vp, vp, vp]),
            "orc_sweep5": (i64, [vp, vp, i64, i32, i64, vp, vp]),
            "orc_canonical5": (u32, [u32]),
            "orc_connected5": (ctypes.c_int, [u32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw64(seed: int, index: int, lane: int, tag: int) -> int:
    return int(lib().orc_draw64(seed, index, lane, tag))


def num_classes(k: int) -> int:
    return int(lib().orc_num_classes(k))


def class_info(k: int):
    nc = num_classes(k)
    canon = np.zeros(nc, dtype=np.uint32)
    mc = np.zeros(nc, dtype=np.int32)
    cm = np.zeros(nc, dtype=np.int32)
    lib().orc_class_info(k, _ptr(canon), _ptr(mc), _ptr(cm))
    return canon, mc, cm


def class_of(k: int, mask: int) -> int:
    return int(lib().orc_class_of(k, mask))


def canonical(k: int, mask: int) -> int:
    return int(lib().orc_canonical(k, mask))


def connected(k: int, mask: int) -> bool:
    return bool(lib().orc_connected(k, mask))


class Graph:
    """Normalised hypergraph held by the oracle (sets of distinct hyperedges)."""

    def __init__(self, members, offsets, num_nodes: int, kmax: int = 4):
        self.members = np.ascontiguousarray(members, dtype=np.int32)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n = int(num_nodes)
        self.kmax = int(kmax)
        self._h = lib().orc_graph_new(_ptr(self.members), _ptr(self.offsets),
                                      self.offsets.shape[0] - 1, self.n, self.kmax)

    @classmethod
    def from_hypergraph(cls, h, kmax: int = 4):
        return cls(h.members, h.offsets, h.num_nodes, kmax)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_graph_free(self._h)
            self._h = None

    def count(self, s: int) -> int:
        return int(lib().orc_graph_count(self._h, s))

    def edges(self, s: int) -> np.ndarray:
        c = self.count(s)
        out = np.zeros((c, s), dtype=np.int32)
        if c:
            lib().orc_graph_edges(self._h, s, _ptr(out))
        return out

    def fill_in(self, k: int, nodes) -> int:
        a = np.ascontiguousarray(nodes, dtype=np.int32)
        return int(lib().orc_fill_in(self._h, k, _ptr(a)))

    def census(self, k: int, threads: int = 1, roots=None):
        """Exact census; returns (hist, number of ESU candidates)."""
        hist = np.zeros(num_classes(k), dtype=np.uint64)
        lo, hi = (0, self.n) if roots is None else roots
        cand = lib().orc_census(self._h, k, threads, lo, hi, _ptr(hist))
        return hist, int(cand)

    def contributions(self, k: int, threads: int = 1) -> np.ndarray:
        rows = sum(self.count(s) for s in range(2, k + 1))
        out = np.zeros((rows, num_classes(k)), dtype=np.uint32)
        sat = lib().orc_contributions(self._h, k, threads, _ptr(out))
        if sat:
            raise OverflowError("per-hyperedge contribution exceeded uint32")
        return out

    def sample_indices(self, s: int, count: int, seed: int, q=None) -> np.ndarray:
        out = np.zeros(count, dtype=np.int64)
        qa = None if q is None else np.ascontiguousarray(q, dtype=np.uint32)
        lib().orc_sample_indices(self._h, s, count, seed, _ptr(qa), _ptr(out))
        return out

    def sample(self, k: int, samples, seed: int, q=None):
        """Alg. 4. samples: dict or list indexed by stratum size. Returns (raw, est, enumerated)."""
        S = np.zeros(k + 1, dtype=np.uint64)
        for s in range(2, k + 1):
            S[s] = samples[s]
        nc = num_classes(k)
        raw = np.zeros(2 * nc, dtype=np.uint64)
        est = np.zeros(nc, dtype=np.float64)
        qa = None if q is None else np.ascontiguousarray(q, dtype=np.uint32)
        e = lib().orc_sample(self._h, k, _ptr(S), seed, _ptr(qa), _ptr(raw), _ptr(est))
        return raw, est, int(e)


def stub_shuffle(members, offsets, seed: int, model: int) -> np.ndarray:
    mem = np.ascontiguousarray(members, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    out = np.zeros_like(mem)
    lib().orc_stub_shuffle(_ptr(mem), _ptr(off), off.shape[0] - 1, seed, model, _ptr(out))
    return out


def config_mcmc(members, offsets, seed: int, model: int, sweeps: int) -> np.ndarray:
    """Configuration-model draw by pairwise reshuffles (see orc_config_mcmc)."""
    mem = np.ascontiguousarray(members, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    out = np.zeros_like(mem)
    lib().orc_config_mcmc(_ptr(mem), _ptr(off), off.shape[0] - 1, seed, model, sweeps, _ptr(out))
    return out


def sample5(members, offsets, num_nodes: int, samples, seed: int, cap: int = 1 << 20):
    """Alg. 4 at order 5 (see orc_sample5): (canonical masks, raw counts, estimates)."""
    mem = np.ascontiguousarray(members, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    S = np.zeros(6, dtype=np.uint64)
    for s in range(2, 6):
        S[s] = samples[s]
    masks = np.zeros(cap, dtype=np.uint32)
    raw = np.zeros(cap, dtype=np.uint64)
    est = np.zeros(cap, dtype=np.float64)
    nc = lib().orc_sample5(_ptr(mem), _ptr(off), off.shape[0] - 1, int(num_nodes), _ptr(S), seed,
                           cap, _ptr(masks), _ptr(raw), _ptr(est))
    nc = min(int(nc), cap)
    return masks[:nc], raw[:nc], est[:nc]


def sweep5(members, offsets, num_nodes: int, cap: int = 1 << 20):
    """Every hyperedge once (see orc_sweep5): (canonical masks, sums)."""
    mem = np.ascontiguousarray(members, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    masks = np.zeros(cap, dtype=np.uint32)
    sums = np.zeros(cap, dtype=np.uint64)
    nc = lib().orc_sweep5(_ptr(mem), _ptr(off), off.shape[0] - 1, int(num_nodes), cap,
                          _ptr(masks), _ptr(sums))
    nc = min(int(nc), cap)
    return masks[:nc], sums[:nc]


def canonical5(mask: int) -> int:
    return int(lib().orc_canonical5(mask))


def connected5(mask: int) -> bool:
    return bool(lib().orc_connected5(mask))
