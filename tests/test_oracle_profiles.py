"""Pins of the profile reference (oracle/profiles.py), CPU only.

* a hand-worked 3-model example (tests/golden/profile_hand.json): the
  abundance and the profile equal the fractions worked out by hand;
* rho / MaxAE / MAE of vectors worked out by hand, rho = +-1 for scaled and
  negated copies, rho equal to scipy's Pearson correlation on random data;
* invariants: unit norm, zeros when the observed counts equal the null mean,
  the sign of over- and under-represented classes;
* a planted mistake (the eps term dropped) fails the hand example.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import profiles as PR
from paper_2209_10241_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hand():
    with open(os.path.join(GOLDEN, "profile_hand.json")) as f:
        return json.load(f)


def test_hand_worked_example():
    h = _hand()
    ab = PR.abundance(h["observed"], h["null_rows"], h["eps"])
    assert np.allclose(ab, [0.0, -1 / 5, 0.0, 10 / 41], rtol=0, atol=1e-15)
    assert np.allclose(ab, h["abundance"], rtol=0, atol=1e-15)
    sp = PR.significance_profile(h["observed"], h["null_rows"], h["eps"])
    want = np.array(h["profile_numer"], dtype=np.float64) / math.sqrt(h["profile_denom_sqrt"])
    assert np.allclose(sp, want, rtol=0, atol=1e-15)


def test_dropping_eps_fails_the_hand_example():
    h = _hand()
    wrong = PR.abundance(h["observed"], h["null_rows"], eps=0.0)
    assert not np.allclose(wrong, h["abundance"], atol=1e-6)


def test_compare_by_hand():
    rho, mx, mae = PR.compare([1, 2, 3, 4], [1, 3, 2, 4])
    assert abs(rho - 0.8) < 1e-15  # dp = dq up to two swapped middles: 4 / 5
    rho, mx, mae = PR.compare([1, 2, 3, 4], [1, 2, 3, 5])
    assert mx == 1.0 and mae == 0.25
    assert abs(PR.compare([1, 2, 3, 4], [2, 4, 6, 8])[0] - 1.0) < 1e-15
    assert abs(PR.compare([1, 2, 3, 4], [-1, -2, -3, -4])[0] + 1.0) < 1e-15
    assert PR.compare([1, 1, 1], [1, 2, 3])[0] == 0.0  # constant profile: rho undefined -> 0


def test_rho_equals_scipy_pearson():
    stats = pytest.importorskip("scipy.stats")
    st = synth.Stream(3, 4)
    for n in (6, 171, 500):
        u = (st.u64(2 * n) >> np.uint64(11)).astype(np.float64) / 2.0 ** 53
        p, q = u[:n], 0.3 * u[:n] + u[n:]
        assert abs(PR.compare(p, q)[0] - stats.pearsonr(p, q)[0]) < 1e-12


def test_profile_invariants():
    st = synth.Stream(5, 6)
    for C, M in ((6, 10), (171, 64)):
        rows = st.below(M * C, 1000).reshape(M, C)
        obs = st.below(C, 2000)
        sp = PR.significance_profile(obs, rows)
        assert abs(np.sum(sp * sp) - 1.0) < 1e-12
        mean = rows.sum(axis=0) / M
        assert np.all(np.sign(sp)[obs > mean] == 1) and np.all(np.sign(sp)[obs < mean] == -1)
    rows = np.array([[3, 5], [5, 7]])
    assert np.all(PR.significance_profile([4, 6], rows) == 0.0)
