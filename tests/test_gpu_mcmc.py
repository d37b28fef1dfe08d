"""GPU parity of the configuration model (pairwise-reshuffle chain) with the oracle.

* hm_configuration_model writes the same members as oracle.config_mcmc, bit
  for bit (same Philox counters, same matching and dealing rules);
* hm_count_null_batch_mcmc rows equal the oracle's census of the oracle's
  own draws, for uneven bases and more than 64 models (several unions);
* a repeated member is rejected with HM_EINVAL.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2209_10241_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,scale,seed,model,sweeps", [
    ("uniform-200", 1.0, 1, 0, 1), ("f2f-330", 0.1, 2, 5, 4), ("coauth-1m", 0.002, 3, 17, 10),
    ("comm-5m", 0.001, 4, 63, 3)])
def test_draw_matches_oracle(hm, name, scale, seed, model, sweeps):
    h = synth.workload(name, seed=seed, scale=scale)
    mem = torch.from_numpy(h.members).cuda()
    off = torch.from_numpy(h.offsets).cuda()
    got = hm.configuration_model(mem, off, h.num_nodes, model, sweeps, seed=99).cpu().numpy()
    want = oracle.config_mcmc(h.members, h.offsets, seed=99, model=model, sweeps=sweeps)
    assert np.array_equal(got, want)


def _oracle_rows(bases, k, J, sweeps, seed):
    rows = []
    for b, h in enumerate(bases):
        for j in range(J):
            t = b * J + j
            mem = oracle.config_mcmc(h.members, h.offsets, seed=seed, model=t, sweeps=sweeps)
            rows.append(oracle.Graph(mem, h.offsets, h.num_nodes, 4).census(
                k, threads=os.cpu_count() or 1)[0])
    return np.array(rows, dtype=np.uint64)


@pytest.mark.parametrize("k", [3, 4])
def test_null_batch_mcmc_matches_oracle(hm, k):
    bases = [synth.workload("f2f-330", seed=1, scale=0.05),
             synth.workload("uniform-200", seed=2, scale=0.3),
             synth.from_edges([[0, 1, 2], [2, 3], [3, 4, 5, 6], [1, 5]], 8)]
    J = 3
    got = hm.null_batch(bases, k, J, seed=21, sweeps=6).cpu().numpy().astype(np.uint64)
    assert (got == _oracle_rows(bases, k, J, 6, 21)).all()


def test_null_batch_mcmc_several_unions(hm):
    bases = [synth.workload("uniform-200", seed=5, scale=0.1),
             synth.workload("f2f-330", seed=6, scale=0.05)]
    J = 40
    got = hm.null_batch(bases, 4, J, seed=8, sweeps=3).cpu().numpy().astype(np.uint64)
    assert (got == _oracle_rows(bases, 4, J, 3, 8)).all()


def test_repeated_member_is_rejected(hm):
    h = synth.from_edges([[0, 1, 1], [2, 3]], 4)
    with pytest.raises(hm.HMError) as e:
        hm.null_batch([h], 4, 2, seed=1, sweeps=2)
    assert e.value.status == 1
