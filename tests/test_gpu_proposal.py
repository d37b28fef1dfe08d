"""GPU parity and behaviour of the learned-proposal path.

* per-hyperedge contributions equal the oracle's bit for bit, and sum to
  countmax_c * T_c (full-sweep identity);
* features equal the CPU reference (float32 vs float64: rtol 1e-5);
* the tensor-core MLP forward and backward equal the float64 reference with
  the same bf16 rounding points, every output and every gradient element
  within its own bound (tests/mlp_bounds.py: float32 accumulation error on
  the sum of |terms|, plus the proven effect of the bf16 roundings that can
  flip), so a small entry cannot be wrong and pass;
* hm_proposal_train equals the chain of calls it wraps bit for bit, and its
  initial weights are the Philox He-uniform draws hm.h states;
* one Adam step equals the reference update;
* training lowers the loss, and the learned proposal's estimates are unbiased
  and bit-exact with the oracle given the same q;
* the trained network gains over uniform sampling: lower mean squared
  relative error at the same number of draws.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import features as F
from oracle import mlp
from paper_2209_10241_gb300 import synth
from tests import mlp_bounds

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("name", ["uniform-200", "tiny"])
def test_contributions_match_oracle(hm, k, name):
    h = (synth.workload("uniform-200") if name == "uniform-200"
         else synth.random_tiny(15, 140, max_size=5, seed=31, dup_frac=0.1))
    g = hm.from_host(h, 4)
    got = hm.contributions(g, k).cpu().numpy().view(np.uint32)
    og = oracle.Graph.from_hypergraph(h, 4)
    want = og.contributions(k, threads=os.cpu_count() or 1)
    assert got.shape == want.shape and (got == want).all()
    hist = hm.count_exact(g, k).cpu().numpy().astype(np.uint64)
    _, _, cm = oracle.class_info(k)
    assert (got.astype(np.uint64).sum(axis=0) == cm.astype(np.uint64) * hist).all()


@pytest.mark.parametrize("k", [3, 4])
def test_features_match_reference(hm, k):
    h = synth.workload("f2f-330", scale=0.2)
    g = hm.from_host(h, 4)
    got = hm.features(g, k).cpu().numpy()
    want = F.features(oracle.Graph.from_hypergraph(h, 4), k)
    assert got.shape == want.shape
    assert np.allclose(got, want, rtol=1e-5, atol=1e-6)


def _mlp_data(n, seed):
    st = synth.Stream(seed, 23)
    u = (st.u64(n * 17) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    X = (u[: n * 16].reshape(n, 16) * 4.0).astype(np.float32)
    X[:, 0] = 1.0
    X[:, 12:] = 0.0
    t = (u[n * 16:] * 4.0 - 2.0).astype(np.float32)
    return X, t


@pytest.mark.parametrize("biases", [False, True])
@pytest.mark.parametrize("n", [1, 17, 1000, 33333])
def test_mlp_forward_backward_match_reference(hm, n, biases):
    p = mlp.init_params(5).copy()
    if biases:  # the initial biases are 0: give them values too
        st = synth.Stream(n, 31)
        for lo, hi in ((mlp.P_B1, mlp.P_W2), (mlp.P_B2, mlp.P_W3), (mlp.P_B3, mlp.NPARAM)):
            u = (st.u64(hi - lo) >> np.uint64(40)).astype(np.float64) / 2 ** 24
            p[lo:hi] = (u - 0.5).astype(np.float32)
    X, t = _mlp_data(n, n)
    dp, dX, dt = (torch.from_numpy(a).cuda() for a in (p, X, t))
    yr, yb, gr, gb, L, Lb = mlp_bounds.bounds(p, X, t)
    # the bounds' reference is the plain float64 reference network
    yr2, _ = mlp.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.array_equal(yr, yr2)
    assert np.allclose(gr, mlp.backward(p.astype(np.float64), X.astype(np.float64),
                                        t.astype(np.float64)), rtol=1e-12, atol=0)
    y = hm.mlp_forward(dp, dX).cpu().numpy().astype(np.float64)
    bad = np.abs(y - yr) > yb
    assert not bad.any(), (np.where(bad)[0][:5], (np.abs(y - yr) / yb)[bad][:5])
    grad, loss = hm.mlp_backward(dp, dX, dt)
    g = grad.cpu().numpy().astype(np.float64)
    bad = np.abs(g - gr) > gb
    assert not bad.any(), (np.where(bad)[0][:5], (np.abs(g - gr) / gb)[bad][:5])
    assert abs(loss.item() - L) <= Lb


def test_adam_step_matches_reference(hm):
    p = mlp.init_params(9)
    st = synth.Stream(9, 2)
    g = ((st.u64(mlp.NPARAM) >> np.uint64(40)).astype(np.float64) / 2 ** 24 - 0.5).astype(np.float32)
    m = np.zeros(mlp.NPARAM, np.float32)
    v = np.zeros(mlp.NPARAM, np.float32)
    dp, dg, dm, dv = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    for step in (1, 2, 3):
        hm.mlp_adam(dp, dg, dm, dv, step, 1e-2)
        p, m, v = mlp.adam_step(p.astype(np.float64), g.astype(np.float64), m, v, step, 1e-2)
    assert np.allclose(dp.cpu().numpy(), p, rtol=1e-5, atol=1e-6)


@pytest.fixture(scope="module")
def trained(hm):
    """Targets from exact contributions on a training instance, and a trained MLP."""
    k = 4
    h = synth.workload("comm-5m", seed=7, scale=0.004)
    g = hm.from_host(h, 4)
    contrib = hm.contributions(g, k)
    exact = hm.count_exact(g, k)
    tgt = hm.proposal_targets(g, k, contrib, exact, eps=1e-9)
    feat = hm.features(g, k)
    p = torch.from_numpy(mlp.init_params(1)).cuda()
    losses = hm.mlp_train(p, feat, tgt, epochs=30, batch=4096, lr=3e-3, seed=3)
    return dict(k=k, params=p, losses=losses, targets=tgt, feat=feat, contrib=contrib,
                exact=exact, g=g, h=h)


def test_backward_and_training_are_deterministic(hm, trained):
    """Fixed-order reductions: the same inputs give the same bits."""
    p = mlp.init_params(5)
    X, t = _mlp_data(33333, 4)
    dp, dX, dt = (torch.from_numpy(a).cuda() for a in (p, X, t))
    g1, l1 = hm.mlp_backward(dp, dX, dt)
    g2, l2 = hm.mlp_backward(dp, dX, dt)
    assert torch.equal(g1, g2) and torch.equal(l1, l2)
    q = torch.from_numpy(mlp.init_params(1)).cuda()
    losses = hm.mlp_train(q, trained["feat"], trained["targets"], epochs=30, batch=4096,
                          lr=3e-3, seed=3)
    assert torch.equal(q, trained["params"])
    assert list(losses) == list(trained["losses"])


def test_training_lowers_the_loss(trained):
    L = trained["losses"]
    assert all(np.isfinite(L)) and L[-1] < 0.5 * L[0], L


def test_targets_match_reference(hm, trained):
    _, _, cm = oracle.class_info(4)
    want = F.targets(trained["contrib"].cpu().numpy().view(np.uint32),
                     trained["exact"].cpu().numpy().astype(np.uint64), cm, 1e-9)
    assert np.allclose(trained["targets"].cpu().numpy(), want, rtol=1e-5, atol=1e-5)


def test_proposal_weights_and_sampler_parity(hm, trained):
    k = 4
    h = synth.workload("comm-5m", seed=8, scale=0.002)
    g = hm.from_host(h, 4)
    q = hm.proposal_weights(g, k, trained["params"], lam=0.1, beta=0.5)
    qn = q.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert (qn >= 1).all()
    # recompute q from the network's outputs: floor boundaries may move by one
    feat = hm.features(g, k)
    y = hm.mlp_forward(trained["params"], feat).cpu().numpy().astype(np.float64)
    y = y - 0.5 * feat.cpu().numpy()[:, 9].astype(np.float64)
    off = 0
    for s in range(2, k + 1):
        n = g.count(s)
        ys = y[off:off + n]
        w = np.exp(ys - ys.max())
        pr = 0.9 * w / w.sum() + 0.1 / n
        want = 1 + np.floor(pr * n * 1024)
        assert np.abs(qn[off:off + n] - want).max() <= 1
        off += n
    # the weighted sampler with the learned q equals the oracle bit for bit
    S = {2: 100, 3: 300, 4: 200}
    est, raw = hm.count_sampled(g, k, samples=S, seed=12, q=q)
    oraw, oest, _ = oracle.Graph.from_hypergraph(h, 4).sample(k, S, seed=12, q=qn.astype(np.uint32))
    assert (raw.cpu().numpy().astype(np.uint64) == oraw).all()
    assert est.cpu().numpy().tobytes() == oest.tobytes()


def test_learned_proposal_gains_over_uniform(hm, trained):
    """Same draws budget, R seeds: mean squared relative error of the class
    estimates (classes with T_c >= 100) is lower with the learned proposal."""
    k = 4
    h = synth.workload("comm-5m", seed=9, scale=0.004)
    g = hm.from_host(h, 4)
    T = hm.count_exact(g, k).cpu().numpy().astype(np.float64)
    q = hm.proposal_weights(g, k, trained["params"], lam=0.1)
    S = {2: 2000, 3: 6000, 4: 4000}
    big = T >= 100
    err = {"uniform": [], "learned": []}
    for r in range(24):
        eu, _ = hm.count_sampled(g, k, samples=S, seed=1000 + r)
        el, _ = hm.count_sampled(g, k, samples=S, seed=1000 + r, q=q)
        for name, e in (("uniform", eu), ("learned", el)):
            e = e.cpu().numpy()
            err[name].append(((e[big] - T[big]) / T[big]) ** 2)
    mse_u = np.mean(err["uniform"])
    mse_l = np.mean(err["learned"])
    assert mse_l < 0.8 * mse_u, (mse_l, mse_u)


def test_mlp_init_is_the_stated_philox_draw(hm):
    seed = 0x1234_5678_9ABC
    got = hm.mlp_init(seed).cpu().numpy()
    want = np.zeros(mlp.NPARAM, dtype=np.float64)
    for lo, hi, fan in ((mlp.P_W1, mlp.P_B1, 16), (mlp.P_W2, mlp.P_B2, 64),
                        (mlp.P_W3, mlp.P_B3, 64)):
        for i in range(lo, hi):
            u = (oracle.draw64(seed, i, 0, 0x494E4954) >> 11) * 2.0 ** -53
            want[i] = (2.0 * u - 1.0) * np.sqrt(6.0 / fan)
    assert np.array_equal(got, want.astype(np.float32))


@pytest.mark.parametrize("k", [3, 4])
def test_proposal_train_equals_the_chain(hm, k):
    h = synth.workload("comm-5m", seed=7, scale=0.002)
    g = hm.from_host(h, 4)
    prop = hm.proposal_train(g, k, seed=11, epochs=6, batch=1024, lr=3e-3)
    assert prop.order == k
    # the five calls it wraps
    contrib = hm.contributions(g, k)
    exact = hm.count_exact(g, k)
    tgt = hm.proposal_targets(g, k, contrib, exact, eps=1e-9)
    feat = hm.features(g, k)
    p = hm.mlp_init(11)
    losses = hm.mlp_train(p, feat, tgt, epochs=6, batch=1024, lr=3e-3, seed=11)
    assert torch.equal(prop.params(), p)
    assert prop.losses == losses
    h2 = synth.workload("comm-5m", seed=8, scale=0.002)
    g2 = hm.from_host(h2, 4)
    q1 = hm.proposal_q(prop, g2, lam=0.1, beta=0.5)
    q2 = hm.proposal_weights(g2, k, p, lam=0.1, beta=0.5)
    assert torch.equal(q1, q2)
    prop.free()


def test_proposal_api_errors(hm):
    h = synth.workload("uniform-200")
    g3 = hm.from_host(h, 3)
    with pytest.raises(hm.HMError) as e:
        hm.proposal_train(g3, 4, seed=1, epochs=1)
    assert e.value.status == 6  # order above the graph's max_order
    with pytest.raises(hm.HMError) as e:
        hm.proposal_train(g3, 3, seed=1, epochs=0)
    assert e.value.status == 1
    prop = hm.proposal_train(hm.from_host(h, 4), 4, seed=1, epochs=1)
    with pytest.raises(hm.HMError) as e:
        hm.proposal_q(prop, g3)  # order-4 proposal on an order-3 graph
    assert e.value.status == 6
