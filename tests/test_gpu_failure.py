"""Failure paths of the C ABI, driven on purpose without faulting the GPU.

* A hash set forced smaller than its key set (the HM_TABLE_CAP test hook):
  every insertion and probe ends after one pass over the slots, and hm_build
  returns HM_ETABLEFULL.
* The bounded device-side waits: hm_selftest_wait runs the sort's look-back
  against a status word that nothing sets; each wait gives up after its poll
  limit and the call returns HM_ETIMEOUT.
After each, the same process builds and counts a graph correctly: the CUDA
context stays usable.
Also: the end-to-end entry point from host buffers (hm_count_exact_host)
against stored oracle histograms.
"""
import json
import os
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2209_10241_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _still_counts(hm):
    h = synth.workload("uniform-200", seed=3, scale=0.5)
    g = hm.from_host(h, 4)
    got = hm.count_exact(g, 4).cpu().numpy().astype(np.uint64)
    want, _ = oracle.Graph.from_hypergraph(h, 4).census(4, threads=os.cpu_count() or 1)
    assert (got == want).all()


@pytest.mark.parametrize("bitmap", ["0", "1"])
def test_undersized_table_returns_etablefull(hm, monkeypatch, bitmap):
    monkeypatch.setenv("HM_PAIR_BITMAP", bitmap)
    monkeypatch.setenv("HM_TABLE_CAP", "16")
    h = synth.workload("uniform-200")
    with pytest.raises(hm.HMError) as e:
        hm.from_host(h, 4)
    assert e.value.status == 4 and "probe bound" in str(e.value)
    monkeypatch.delenv("HM_TABLE_CAP")
    _still_counts(hm)


def test_bounded_wait_returns_etimeout(hm):
    t0 = time.monotonic()
    with pytest.raises(hm.HMError) as e:
        hm.selftest_wait()
    assert e.value.status == 5 and "gave up" in str(e.value)
    assert time.monotonic() - t0 < 60
    _still_counts(hm)
    # the timeout count was cleared: a normal build reports no timeout
    _still_counts(hm)


@pytest.mark.parametrize("case", ["f2f-330", "coauth-1m-s001"])
@pytest.mark.parametrize("k", [3, 4])
def test_exact_host_against_stored_oracle(hm, case, k):
    with open(os.path.join(GOLDEN, f"census_{case}.json")) as f:
        rec = json.load(f)
    h = synth.workload(rec["workload"], seed=rec["seed"], scale=rec["scale"])
    mem = torch.from_numpy(h.members).pin_memory()
    off = torch.from_numpy(h.offsets).pin_memory()
    out = hm.count_exact_host(mem, off, h.num_nodes, k)
    assert out.numpy().astype(np.uint64).tolist() == rec["hist"][str(k)]
    # pageable host buffers work too
    out2 = hm.count_exact_host(torch.from_numpy(h.members), torch.from_numpy(h.offsets),
                               h.num_nodes, k)
    assert torch.equal(out, out2)
