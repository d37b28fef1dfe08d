"""Thin ctypes binding of libhm.so (argument marshalling only).

Every computation runs in the CUDA library; this module passes torch device
pointers and the current CUDA stream to the C ABI declared in include/hm.h.
If the library is missing, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhm.so")
_lib = None

HM_OK = 0
_STATUS = {1: "HM_EINVAL", 2: "HM_ENOMEM", 3: "HM_ECUDA", 4: "HM_ETABLEFULL",
           5: "HM_ETIMEOUT", 6: "HM_EUNSUPPORTED"}


class HMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_vp = ctypes.c_void_p
_SIGS = {
    "hm_last_error": (ctypes.c_char_p, []),
    "hm_version": (ctypes.c_char_p, []),
    "hm_num_classes": (ctypes.c_int, [ctypes.c_int]),
    "hm_class_info": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
    "hm_class_of_mask": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, _vp]),
    "hm_build": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, _vp,
                                ctypes.POINTER(_vp)]),
    "hm_graph_info": (ctypes.c_int, [_vp, _vp]),
    "hm_graph_edges": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "hm_count_exact": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "hm_count_sampled": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_uint64, ctypes.c_uint64,
                                        _vp, _vp, _vp, _vp]),
    "hm_count_sampled_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_uint64,
                                                ctypes.c_uint64, _vp, _vp, _vp, _vp]),
    "hm_count_null_batch": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_uint64, _vp, _vp]),
    "hm_count_null_batch_mcmc": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                _vp, _vp]),
    "hm_configuration_model": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64,
                                              _vp, _vp]),
    "hm_contributions": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "hm_features": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "hm_mlp_num_params": (ctypes.c_int, []),
    "hm_mlp_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "hm_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp]),
    "hm_mlp_backward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp]),
    "hm_mlp_adam": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, _vp]),
    "hm_mlp_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                    ctypes.c_float, ctypes.c_uint64, _vp, _vp]),
    "hm_proposal_targets": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_float, _vp, _vp]),
    "hm_proposal_weights_params": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_float,
                                                  ctypes.c_float, _vp, _vp]),
    "hm_mlp_init": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp]),
    "hm_proposal_train": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.c_int64, ctypes.c_float, _vp, _vp,
                                         ctypes.POINTER(_vp)]),
    "hm_proposal_params": (ctypes.c_int, [_vp, _vp, _vp]),
    "hm_proposal_order": (ctypes.c_int, [_vp]),
    "hm_proposal_weights": (ctypes.c_int, [_vp, _vp, ctypes.c_float, ctypes.c_float, _vp, _vp]),
    "hm_proposal_free": (None, [_vp]),
    "hm_count_exact_host": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int,
                                           _vp, _vp]),
    "hm_work_totals": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "hm_count_exact_baseline": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32,
                                               ctypes.c_int, _vp, _vp, _vp]),
    "hm_count_sampled5": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32, _vp,
                                         ctypes.c_uint64, ctypes.c_uint64, _vp, _vp, _vp,
                                         ctypes.c_int64, _vp, _vp]),
    "hm_trace_enable": (ctypes.c_int, [ctypes.c_int]),
    "hm_trace_only": (ctypes.c_int, [ctypes.c_char_p]),
    "hm_launch_count": (ctypes.c_uint64, []),
    "hm_l2_read_bandwidth": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, _vp, _vp]),
    "hm_selftest_wait": (ctypes.c_int, [_vp]),
    "hm_debug_canonical_check": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "hm_serialize_launches": (ctypes.c_int, [ctypes.c_int]),
    "hm_significance_profile": (ctypes.c_int, [ctypes.c_int, _vp, _vp, ctypes.c_int,
                                               ctypes.c_double, _vp, _vp, _vp]),
    "hm_profile_compare": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _vp]),
    "hm_counts_to_double": (ctypes.c_int, [_vp, ctypes.c_int64, _vp, _vp]),
    "hm_trace_read": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.c_int, _vp, _vp]),
    "hm_free": (None, [_vp]),
}
# declared in include/hm.h; checked by the ABI test
EXPORTS = tuple(_SIGS)


def load(path: str = LIB_PATH):
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -m paper_2209_10241_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != HM_OK:
        raise HMError(status, load().hm_last_error().decode())


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream, device=None):
    """The CUDA stream handle to pass: `stream`, else the current stream of
    `device` (a tensor's device index; the current device when None). The raw
    query skips building a torch Stream object, a few microseconds per call."""
    if stream is None:
        if _raw_stream is not None:
            return ctypes.c_void_p(_raw_stream(torch.cuda.current_device() if device is None
                                               else device))
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def num_classes(order: int) -> int:
    return int(load().hm_num_classes(order))


def class_info(order: int, cls: int):
    m, a, b = ctypes.c_uint32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().hm_class_info(order, cls, ctypes.byref(m), ctypes.byref(a), ctypes.byref(b)))
    return m.value, a.value, b.value


def class_of_mask(order: int, mask: int) -> int:
    c = ctypes.c_int32()
    _check(load().hm_class_of_mask(order, mask, ctypes.byref(c)))
    return c.value


class Graph:
    """A hypergraph built on the current CUDA device (hm_build)."""

    def __init__(self, handle, kmax: int):
        self._h = handle
        self.kmax = kmax
        self._counts = None

    @property
    def counts(self):
        """[nodes, input hyperedges, |E_2|, |E_3|, |E_4|, oversized, 0, 0]
        (hm_graph_info, read on first use)."""
        if self._counts is None:
            if not getattr(self, "_h", None):
                raise RuntimeError("graph already freed")
            counts = (ctypes.c_int64 * 8)()
            _check(load().hm_graph_info(self._h, counts))
            self._counts = list(counts)
        return self._counts

    @property
    def num_nodes(self):
        return self.counts[0]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hm_free(self._h)
            self._h = None

    def free(self):
        """Releases the device structures; the counts stay readable."""
        if getattr(self, "_h", None) and self._counts is None:
            self.counts
        self.__del__()

    def count(self, s: int) -> int:
        return int(self.counts[s])

    def edges(self, s: int, stream=None) -> torch.Tensor:
        out = torch.empty((self.count(s), s), dtype=torch.int32, device="cuda")
        _check(load().hm_graph_edges(self._h, s, _dptr(out), _stream(stream)))
        return out


def build(members: torch.Tensor, offsets: torch.Tensor, num_nodes: int, max_order: int = 4,
          stream=None) -> Graph:
    """hm_build on device tensors (int32 members, int64 offsets)."""
    assert members.is_cuda and offsets.is_cuda
    if members.dtype != torch.int32 or not members.is_contiguous():
        members = members.contiguous().to(torch.int32)
    if offsets.dtype != torch.int64 or not offsets.is_contiguous():
        offsets = offsets.contiguous().to(torch.int64)
    h = ctypes.c_void_p()
    _check(load().hm_build(_dptr(members), _dptr(offsets), offsets.numel() - 1, int(num_nodes),
                           int(max_order), _stream(stream, members.device.index), ctypes.byref(h)))
    return Graph(h, max_order)


def count_exact(g: Graph, order: int, out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """hm_count_exact; returns an int64 device tensor holding the uint64 counts."""
    if out is None:
        out = torch.empty(max(1, num_classes(order)), dtype=torch.int64, device="cuda")
    _check(load().hm_count_exact(g._h, order, _dptr(out), _stream(stream, out.device.index)))
    return out


def count_sampled(g: Graph, order: int, samples=None, total: int = 0, seed: int = 0,
                  q: torch.Tensor = None, stream=None):
    """hm_count_sampled; returns (estimates float64, raw int64[2*ncls]) device tensors."""
    nc = max(1, num_classes(order))
    est = torch.empty(nc, dtype=torch.float64, device="cuda")
    raw = torch.empty(2 * nc, dtype=torch.int64, device="cuda")
    sp = None
    if samples is not None:
        arr = (ctypes.c_uint64 * 5)()
        for s in range(2, min(order, 4) + 1):
            arr[s] = int(samples[s])
        sp = arr
    _check(load().hm_count_sampled(g._h, order, sp, int(total), int(seed) & (2**64 - 1),
                                   _dptr(q), _dptr(est), _dptr(raw), _stream(stream)))
    return est, raw


def count_sampled_noalloc(g: Graph, order: int, est: torch.Tensor, raw: torch.Tensor = None,
                          samples=None, total: int = 0, seed: int = 0, q: torch.Tensor = None,
                          stream=None):
    """hm_count_sampled_noalloc into caller-provided device buffers (allocates nothing)."""
    sp = None
    if samples is not None:
        arr = (ctypes.c_uint64 * 5)()
        for s in range(2, min(order, 4) + 1):
            arr[s] = int(samples[s])
        sp = arr
    _check(load().hm_count_sampled_noalloc(g._h, order, sp, int(total), int(seed) & (2**64 - 1),
                                           _dptr(q), _dptr(est), _dptr(raw), _stream(stream)))
    return est, raw


def null_batch(bases, order: int, models_per_base: int, seed: int, stream=None,
               sweeps: int = None) -> torch.Tensor:
    """hm_count_null_batch (stub shuffling), or hm_count_null_batch_mcmc when
    `sweeps` is given (the configuration model by pairwise reshuffles), over
    host hypergraphs (synth.Hypergraph); returns an int64 device tensor
    [len(bases) * models_per_base, ncls] of uint64 counts."""
    import numpy as np
    mem = np.concatenate([b.members for b in bases]) if bases else np.zeros(0, np.int32)
    offs, edges, shift = [np.zeros(1, np.int64)], [0], 0
    for b in bases:
        offs.append(b.offsets[1:] + shift)
        shift += int(b.offsets[-1])
        edges.append(edges[-1] + b.num_hyperedges)
    off = np.concatenate(offs)
    dmem = torch.from_numpy(mem.astype(np.int32)).cuda()
    doff = torch.from_numpy(off.astype(np.int64)).cuda()
    hedges = (ctypes.c_int64 * len(edges))(*edges)
    hn = (ctypes.c_int32 * len(bases))(*[b.num_nodes for b in bases])
    nc = num_classes(order)
    out = torch.empty((len(bases) * models_per_base, max(1, nc)), dtype=torch.int64, device="cuda")
    if sweeps is None:
        _check(load().hm_count_null_batch(len(bases), _dptr(dmem), _dptr(doff), hedges, hn,
                                          order, models_per_base, int(seed) & (2**64 - 1),
                                          _dptr(out), _stream(stream)))
    else:
        _check(load().hm_count_null_batch_mcmc(len(bases), _dptr(dmem), _dptr(doff), hedges, hn,
                                               order, models_per_base, int(sweeps),
                                               int(seed) & (2**64 - 1), _dptr(out),
                                               _stream(stream)))
    return out


def configuration_model(members: torch.Tensor, offsets: torch.Tensor, num_nodes: int,
                        model: int, sweeps: int, seed: int, stream=None) -> torch.Tensor:
    """hm_configuration_model: one draw's members (int32 device tensor, the
    offsets stay those of the input)."""
    out = torch.empty_like(members)
    _check(load().hm_configuration_model(_dptr(members), _dptr(offsets), offsets.numel() - 1,
                                         int(num_nodes), int(model), int(sweeps),
                                         int(seed) & (2**64 - 1), _dptr(out), _stream(stream)))
    return out


def from_host(h, max_order: int = 4, device="cuda") -> Graph:
    """Copy a synth.Hypergraph to the device and build it."""
    mem = torch.from_numpy(h.members).to(device)
    off = torch.from_numpy(h.offsets).to(device)
    return build(mem, off, h.num_nodes, max_order)


def count_exact_host(members, offsets, num_nodes: int, order: int, out=None, stream=None):
    """hm_count_exact_host on host (ideally pinned) tensors; returns a host int64 tensor."""
    assert not members.is_cuda and not offsets.is_cuda
    if out is None:
        out = torch.empty(num_classes(order), dtype=torch.int64)
    _check(load().hm_count_exact_host(_dptr(members), _dptr(offsets), offsets.numel() - 1,
                                      int(num_nodes), int(order), _dptr(out), _stream(stream)))
    return out


def trace_enable(on: bool = True):
    _check(load().hm_trace_enable(1 if on else 0))


def trace_only(name: str = None):
    """Trace only the spans named `name` (None = every span)."""
    _check(load().hm_trace_only(name.encode() if name else None))


def trace_read(max_entries: int = 4096):
    """[(kernel name, ms)] recorded since the last read."""
    name_len = 32
    names = ctypes.create_string_buffer(max_entries * name_len)
    ms = (ctypes.c_float * max_entries)()
    cnt = ctypes.c_int()
    _check(load().hm_trace_read(max_entries, names, name_len, ms, ctypes.byref(cnt)))
    raw = names.raw
    return [(raw[i * name_len:(i + 1) * name_len].split(b"\0")[0].decode(), float(ms[i]))
            for i in range(cnt.value)]


FAMILIES = {3: ("census_T3", "census_W", "census_Wb", "uses_Wb"),
            4: ("census_Q", "census_TX", "census_S", "census_P", "census_Sb", "census_Pb",
                "uses_Sb", "uses_Pb", "census_TXb", "uses_TXb")}


def work_totals(g: Graph, order: int, stream=None) -> dict:
    """Index-space sizes of the exact census {kernel name: items} (see hm.h)."""
    arr = (ctypes.c_uint64 * 10)()
    _check(load().hm_work_totals(g._h, order, arr, _stream(stream)))
    return {name: int(arr[i]) for i, name in enumerate(FAMILIES[order])}


def selftest_wait(stream=None):
    """hm_selftest_wait: raises HMError (HM_ETIMEOUT when the bounded waits work)."""
    _check(load().hm_selftest_wait(_stream(stream)))


def serialize_launches(on: bool = True):
    """hm_serialize_launches: forked work in order on the calling stream."""
    _check(load().hm_serialize_launches(1 if on else 0))


def launch_count() -> int:
    """Kernels launched by libhm.so so far in this process."""
    return int(load().hm_launch_count())


def l2_read_bandwidth(nbytes: int = 64 << 20, reps: int = 20, stream=None) -> float:
    """hm_l2_read_bandwidth: GB/s of reads from an L2-resident buffer."""
    out = ctypes.c_double(0.0)
    _check(load().hm_l2_read_bandwidth(nbytes, reps, ctypes.byref(out), _stream(stream)))
    return out.value


def _rows(g: Graph, order: int) -> int:
    return sum(g.count(s) for s in range(2, order + 1))


def contributions(g: Graph, order: int, stream=None) -> torch.Tensor:
    """hm_contributions: int32 device tensor [rows, ncls] holding the uint32 counts n_{e,c}."""
    out = torch.empty((_rows(g, order), num_classes(order)), dtype=torch.int32, device="cuda")
    _check(load().hm_contributions(g._h, order, _dptr(out), _stream(stream)))
    return out


def features(g: Graph, order: int, stream=None) -> torch.Tensor:
    """hm_features: float32 device tensor [rows, 16]."""
    out = torch.empty((_rows(g, order), 16), dtype=torch.float32, device="cuda")
    _check(load().hm_features(g._h, order, _dptr(out), _stream(stream)))
    return out


def mlp_num_params() -> int:
    return int(load().hm_mlp_num_params())


def mlp_forward(params: torch.Tensor, x: torch.Tensor, stream=None) -> torch.Tensor:
    y = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    _check(load().hm_mlp_forward(_dptr(params), _dptr(x), x.shape[0], _dptr(y), _stream(stream)))
    return y


def mlp_backward(params: torch.Tensor, x: torch.Tensor, target: torch.Tensor, stream=None):
    """Gradient of mean((y - target)^2); returns (grad float32[P], sum of squared errors)."""
    n = x.shape[0]
    grad = torch.empty(mlp_num_params(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(max(1, load().hm_mlp_scratch_bytes(n)), dtype=torch.uint8,
                          device="cuda")
    _check(load().hm_mlp_backward(_dptr(params), _dptr(x), _dptr(target), n, _dptr(grad),
                                  _dptr(loss), _dptr(scratch), _stream(stream)))
    return grad, loss


def mlp_adam(params, grad, m, v, step: int, lr: float, stream=None):
    _check(load().hm_mlp_adam(_dptr(params), _dptr(grad), _dptr(m), _dptr(v), int(step),
                              float(lr), _stream(stream)))


def mlp_train(params: torch.Tensor, x: torch.Tensor, target: torch.Tensor, epochs: int,
              batch: int = 8192, lr: float = 1e-3, seed: int = 0, stream=None):
    """hm_mlp_train in place on params; returns the mean loss of every epoch."""
    losses = (ctypes.c_float * max(1, epochs))()
    _check(load().hm_mlp_train(_dptr(params), _dptr(x), _dptr(target), x.shape[0], int(epochs),
                               int(batch), float(lr), int(seed) & (2**64 - 1), losses,
                               _stream(stream)))
    return [float(losses[i]) for i in range(epochs)]


def proposal_targets(g: Graph, order: int, contrib: torch.Tensor, exact: torch.Tensor,
                     eps: float = 1e-9, stream=None) -> torch.Tensor:
    out = torch.empty(contrib.shape[0], dtype=torch.float32, device="cuda")
    _check(load().hm_proposal_targets(g._h, order, _dptr(contrib), _dptr(exact), float(eps),
                                      _dptr(out), _stream(stream)))
    return out


def proposal_weights(g: Graph, order: int, params: torch.Tensor, lam: float = 0.1,
                     beta: float = 0.0, stream=None) -> torch.Tensor:
    """hm_proposal_weights_params: integer proposal q (int32 tensor holding
    uint32) for hm_count_sampled from explicit MLP parameters."""
    q = torch.empty(_rows(g, order), dtype=torch.int32, device="cuda")
    _check(load().hm_proposal_weights_params(g._h, order, _dptr(params), float(lam),
                                             float(beta), _dptr(q), _stream(stream)))
    return q


def mlp_init(seed: int, stream=None) -> torch.Tensor:
    """hm_mlp_init: He-uniform initial parameters from Philox(seed)."""
    p = torch.empty(mlp_num_params(), dtype=torch.float32, device="cuda")
    _check(load().hm_mlp_init(_dptr(p), int(seed) & (2**64 - 1), _stream(stream)))
    return p


class Proposal:
    """Owning handle of a trained proposal (hm_proposal)."""

    def __init__(self, handle, losses):
        self._h = handle
        self.losses = losses

    @property
    def order(self) -> int:
        return int(load().hm_proposal_order(self._h))

    def params(self, stream=None) -> torch.Tensor:
        out = torch.empty(mlp_num_params(), dtype=torch.float32, device="cuda")
        _check(load().hm_proposal_params(self._h, _dptr(out), _stream(stream)))
        return out

    def free(self):
        if self._h:
            load().hm_proposal_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def proposal_train(train: Graph, order: int, seed: int = 0, epochs: int = 300,
                   batch: int = 8192, lr: float = 1e-3, stream=None) -> Proposal:
    """hm_proposal_train on a built graph; returns the Proposal handle (with the
    per-epoch mean losses in .losses)."""
    losses = (ctypes.c_float * max(1, epochs))()
    h = _vp()
    _check(load().hm_proposal_train(train._h, order, int(seed) & (2**64 - 1), int(epochs),
                                    int(batch), float(lr), losses, _stream(stream),
                                    ctypes.byref(h)))
    return Proposal(h, [float(losses[i]) for i in range(epochs)])


def proposal_q(p: Proposal, g: Graph, lam: float = 0.1, beta: float = 0.0,
               stream=None) -> torch.Tensor:
    """hm_proposal_weights: integer proposal q of graph g from a trained proposal."""
    q = torch.empty(_rows(g, p.order), dtype=torch.int32, device="cuda")
    _check(load().hm_proposal_weights(p._h, g._h, float(lam), float(beta), _dptr(q),
                                      _stream(stream)))
    return q


def counts_to_double(counts: torch.Tensor, stream=None) -> torch.Tensor:
    """hm_counts_to_double on a device tensor of uint64 counts (held as int64)."""
    out = torch.empty(counts.numel(), dtype=torch.float64, device="cuda")
    _check(load().hm_counts_to_double(_dptr(counts), counts.numel(), _dptr(out),
                                      _stream(stream)))
    return out


def significance_profile(observed: torch.Tensor, null_rows: torch.Tensor, eps: float = 4.0,
                         stream=None):
    """hm_significance_profile: (profile, abundance) float64 device tensors.
    observed: float64 [C] (or int64 counts, converted on the device);
    null_rows: int64 [M, C] holding uint64 counts."""
    if observed.dtype != torch.float64:
        observed = counts_to_double(observed, stream)
    M, C = null_rows.shape
    prof = torch.empty(C, dtype=torch.float64, device="cuda")
    ab = torch.empty(C, dtype=torch.float64, device="cuda")
    _check(load().hm_significance_profile(int(C), _dptr(observed), _dptr(null_rows), int(M),
                                          float(eps), _dptr(prof), _dptr(ab), _stream(stream)))
    return prof, ab


def profile_compare(estimated: torch.Tensor, exact: torch.Tensor, stream=None) -> torch.Tensor:
    """hm_profile_compare: float64 device tensor (rho, MaxAE, MAE)."""
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    _check(load().hm_profile_compare(int(exact.numel()), _dptr(estimated), _dptr(exact),
                                     _dptr(out), _stream(stream)))
    return out


def count_exact_baseline(members: torch.Tensor, offsets: torch.Tensor, num_nodes: int,
                         order: int, stream=None):
    """hm_count_exact_baseline (Alg. 1 on the GPU): (hist int64 device tensor,
    candidates generated, distinct projection pairs)."""
    nc = num_classes(order)
    out = torch.empty(nc, dtype=torch.int64, device="cuda")
    info = (ctypes.c_uint64 * 2)()
    _check(load().hm_count_exact_baseline(_dptr(members), _dptr(offsets), offsets.numel() - 1,
                                          int(num_nodes), int(order), _dptr(out), info,
                                          _stream(stream)))
    return out, int(info[0]), int(info[1])


def count_sampled5(members: torch.Tensor, offsets: torch.Tensor, num_nodes: int, samples=None,
                   total: int = 0, seed: int = 0, capacity: int = 1 << 20, stream=None):
    """hm_count_sampled5 (Alg. 4 at order 5): (canonical masks int64, raw
    counts int64, estimates float64) device tensors of the classes met,
    ascending by mask."""
    arr = None
    if samples is not None:
        arr = (ctypes.c_uint64 * 6)(*[int(samples.get(s, 0)) if isinstance(samples, dict)
                                      else int(samples[s]) for s in range(6)])
    masks = torch.empty(capacity, dtype=torch.int32, device="cuda")
    raw = torch.empty(capacity, dtype=torch.int64, device="cuda")
    est = torch.empty(capacity, dtype=torch.float64, device="cuda")
    nc = ctypes.c_int64()
    _check(load().hm_count_sampled5(_dptr(members), _dptr(offsets), offsets.numel() - 1,
                                    int(num_nodes), arr, int(total), int(seed) & (2**64 - 1),
                                    _dptr(masks), _dptr(raw), _dptr(est), int(capacity),
                                    ctypes.byref(nc), _stream(stream)))
    k = min(int(nc.value), capacity)
    return masks[:k].to(torch.int64) & 0xFFFFFFFF, raw[:k], est[:k]


def debug_canonical_check(g: Graph, order: int, stream=None):
    """hm_debug_canonical_check: (sets emitted, repeated keys)."""
    out = (ctypes.c_uint64 * 2)()
    _check(load().hm_debug_canonical_check(g._h, order, out, _stream(stream)))
    return int(out[0]), int(out[1])
