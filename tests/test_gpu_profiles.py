"""GPU parity of the motif significance profile and its comparison metrics
(hm_significance_profile, hm_profile_compare) with the oracle (oracle/profiles.py).

Double precision with sums in another order than numpy's: every value within
1e-12 relative (a sum of at most 171 terms errs by < 200 ulp).
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import profiles as PR
from paper_2209_10241_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _close(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.all(np.abs(a - b) <= 1e-12 * np.maximum(1.0, np.abs(b)))


def test_hand_worked_example(hm):
    with open(os.path.join(GOLDEN, "profile_hand.json")) as f:
        h = json.load(f)
    obs = torch.tensor(h["observed"], dtype=torch.float64, device="cuda")
    rows = torch.tensor(h["null_rows"], dtype=torch.int64, device="cuda")
    sp, ab = hm.significance_profile(obs, rows, eps=h["eps"])
    want = np.array(h["profile_numer"], np.float64) / np.sqrt(h["profile_denom_sqrt"])
    assert _close(sp.cpu().numpy(), want) and _close(ab.cpu().numpy(), h["abundance"])


@pytest.mark.parametrize("k", [3, 4])
def test_profile_of_a_null_batch_matches_oracle(hm, k):
    h = synth.workload("f2f-330", seed=2, scale=0.1)
    M = 10
    rows = hm.null_batch([h], k, M, seed=9)
    obs = hm.count_exact(hm.from_host(h, 4), k)
    sp, ab = hm.significance_profile(obs, rows)
    # the oracle side: its own census of the base and of its own stub shuffles
    og = oracle.Graph.from_hypergraph(h, 4)
    o_obs = og.census(k, threads=os.cpu_count() or 1)[0]
    o_rows = np.array([oracle.Graph(oracle.stub_shuffle(h.members, h.offsets, seed=9, model=t),
                                    h.offsets, h.num_nodes, 4).census(k)[0] for t in range(M)])
    assert _close(sp.cpu().numpy(), PR.significance_profile(o_obs, o_rows))
    assert _close(ab.cpu().numpy(), PR.abundance(o_obs, o_rows))
    # an estimated profile against the exact one
    est, _ = hm.count_sampled(hm.from_host(h, 4), k, total=3000, seed=4)
    sp_hat, _ = hm.significance_profile(est, rows)
    got = hm.profile_compare(sp_hat, sp).cpu().numpy()
    want = PR.compare(sp_hat.cpu().numpy(), sp.cpu().numpy())
    assert _close(got, want)


@pytest.mark.parametrize("C", [1, 6, 171, 300])
def test_compare_matches_oracle(hm, C):
    st = synth.Stream(C, 8)
    u = (st.u64(2 * C) >> np.uint64(11)).astype(np.float64) / 2.0 ** 53 - 0.5
    p, q = torch.from_numpy(u[:C]).cuda(), torch.from_numpy(0.5 * u[:C] + u[C:]).cuda()
    assert _close(hm.profile_compare(p, q).cpu().numpy(), PR.compare(p.cpu().numpy(),
                                                                     q.cpu().numpy()))


def test_profile_errors(hm):
    obs = torch.zeros(4, dtype=torch.float64, device="cuda")
    rows = torch.zeros((2, 4), dtype=torch.int64, device="cuda")
    with pytest.raises(hm.HMError) as e:
        hm.significance_profile(obs, rows, eps=-1.0)
    assert e.value.status == 1
    sp, _ = hm.significance_profile(obs, rows)
    assert torch.count_nonzero(sp).item() == 0
