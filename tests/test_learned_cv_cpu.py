"""Host pieces of the learned control variate: the remaining-contract
program of a state and the network feature rows.

* from inception (k = 0, no knock-in) the state program pays exactly what
  the worst-of autocall workload pays, path by path on the oracle;
* from a later state it pays what the term sheet says (coupon index shifted
  by the elapsed dates, knock-in flag carried), written out by hand;
* the feature rows equal the oracle's layout.
"""
import numpy as np
import pytest

import workloads as W
from oracle import cv, il_text, mc
from oracle.paths import Market, simulate
from paper_2108_03076_gb300 import learned_cv as L

MK = Market([1.0, 1.0, 1.0], [0.25, 0.2, 0.3], W.const_corr(3, 0.5), 0.03,
            [365, 730, 1095, 1460, 1825])


def test_inception_state_is_the_workload_contract():
    a = mc.payoffs(il_text.parse(L.autocall_state_text(5, 0, 0.05, 1.0, 0.6, False)), MK, {}, 0, 1,
                   4096, 3)
    b = mc.payoffs(il_text.parse(W.autocall_text([1.0, 1.0, 1.0], 5)), MK, {}, 0, 1, 4096, 3)
    np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("k,flag", [(2, False), (2, True), (4, False), (4, True)])
def test_later_state_pays_the_term_sheet(k, flag):
    n_rem = 5 - k
    mk = Market([0.9, 1.1, 0.8], [0.25, 0.2, 0.3], W.const_corr(3, 0.5), 0.02,
                [365 * (j + 1) for j in range(n_rem)])
    cpn, call, kil = 0.06, 1.02, 0.55
    got = mc.payoffs(il_text.parse(L.autocall_state_text(n_rem, k, cpn, call, kil, flag)), mk, {}, 0, 1,
                     4096, 5)
    S = np.moveaxis(simulate(mk, 5, 0, np.arange(4096)), 1, 2)
    worst = S.min(axis=2)

    def by_hand(p):
        for j in range(1, n_rem + 1):
            if worst[p, j] >= call:
                return (1 + cpn * (k + j)) * mk.disc(j)
        ki = flag or any(worst[p, j] <= kil for j in range(1, n_rem + 1))
        return (worst[p, n_rem] if ki else 1.0) * mk.disc(n_rem)

    np.testing.assert_allclose(got, [by_hand(p) for p in range(4096)], rtol=1e-13, atol=1e-15)


def test_feature_rows_match_the_oracle_layout():
    rng = np.random.default_rng(0)
    lnS = rng.normal(size=(7, 3))
    ki = rng.uniform(size=7) < 0.5
    sig = [0.2, 0.25, 0.3]
    got = L.features(lnS, ki, np.full(7, 2), 5, np.array(sig)[None, :], 0.5, 0.03, np.ones(7), 0.05, 1.0, 0.6)
    want = cv.autocall_features(lnS, ki, 2, 5, sig, 0.5, 0.03, 1.0, 0.05, 1.0, 0.6)
    np.testing.assert_allclose(got, want, rtol=0, atol=0)


def test_sampled_states_are_reachable():
    st = L.sample_states(2000, np.random.default_rng(1))
    worst = np.exp(st["lnS"]).min(1)
    later = st["k"] >= 1
    assert np.all(worst[later] < st["call"][later])
    assert np.all(st["ki"][later & (worst <= st["kil"])])
    assert not np.any(st["ki"][~later])
    assert set(np.unique(st["k"])) == {0, 1, 2, 3, 4}
