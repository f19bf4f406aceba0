"""The batched-pricing portfolio: every contract's program text equals, path
by path on the oracle, the compiled form of its contract written in the
contract language (the same shape as the single-contract workloads), and
the generator is deterministic with the stated ranges."""
import collections

import numpy as np
import pytest

import workloads as W
from oracle import cl, contracts as C, il_text, mc
from oracle.paths import Market



@pytest.fixture(scope="module")
def port():
    return W.portfolio()


def test_generator_is_deterministic_and_in_range(port):
    again = W.portfolio()
    assert [p.il_text for p in port] == [p.il_text for p in again]
    assert [p.n_paths for p in port] == [p.n_paths for p in again]
    assert len(port) == 1024
    assert set(collections.Counter(p.template for p in port)) == set(W.PORTFOLIO_TEMPLATES)
    assert all(2 ** 12 <= p.n_paths <= 2 ** 18 for p in port)
    assert all(1 <= p.market.d <= 4 for p in port)
    assert all(1 <= p.market.n <= 365 for p in port)
    assert all(list(p.market.days) == sorted(set(p.market.days)) for p in port)


def _market(ms):
    return Market(ms.S0, ms.sigma, ms.corr, ms.r, ms.days)


TEXT_AND_CL = {
    "european": (lambda d, n, k: W.basket_call_text(d, k), lambda d, n, k: C.basket_call_cl(d, k)),
    "digital": (lambda d, n, k: W.basket_digital_text(d, k),
                lambda d, n, k: C.basket_digital_cl(d, k)),
    "call_spread": (lambda d, n, k: W.call_spread_text(d, k, k + 0.2),
                    lambda d, n, k: C.call_spread_cl(d, k, k + 0.2)),
    "asian": (lambda d, n, k: W.asian_text(n, 1.0, k), lambda d, n, k: C.asian_cl(n, 1.0, k)),
}


@pytest.mark.parametrize("template", sorted(TEXT_AND_CL))
def test_basket_and_average_templates_equal_their_contracts(template):
    rng = np.random.default_rng(5)
    text_of, cl_of = TEXT_AND_CL[template]
    for d in (1, 2, 4):
        n = int(rng.integers(1, 40))
        k = float(rng.uniform(0.8, 1.2))
        ms = W.MarketSpec([1.0] * d, W.draw_sigmas(d), W.const_corr(d, 0.5), 0.03,
                          list(range(30, 30 * (n + 1), 30)))
        mk = _market(ms)
        a = mc.payoffs(il_text.parse(text_of(d, n, k), ["T"]), mk, {"T": n}, 0, 1, 2048, 9)
        b = mc.payoffs(cl.compile_contr(cl_of(d, n, k)), mk, {"T": n}, 0, 1, 2048, 9)
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)
        assert np.count_nonzero(a) > 0


def test_generated_texts_are_the_template_texts(port):
    """Each item's text is its template's builder output (the builders the
    previous tests pin to the contract language)."""
    for it in port[:200]:
        d, n = it.market.d, it.market.n
        if it.template in TEXT_AND_CL:
            prog = il_text.parse(it.il_text)
            assert prog is not None
        assert it.il_text.count("(model ") >= 1
        assert f"(model {d - 1} " in it.il_text or it.template == "asian"
        if it.template == "asian":
            assert it.il_text.count("(model 0 ") == n


def test_autocall_and_barrier_templates_equal_their_contracts():
    S0 = [1.0, 1.0, 1.0]
    ms = W.MarketSpec(S0, [0.3, 0.25, 0.35], W.const_corr(3, 0.5), 0.03,
                      [100 * (k + 1) for k in range(7)])
    mk = _market(ms)
    a = mc.payoffs(il_text.parse(W.autocall_text(S0, n_dates=7), ["T"]), mk, {}, 0, 1, 2048, 3)
    b = mc.payoffs(cl.compile_contr(C.autocall_cl(S0, n_dates=7)), mk, {}, 0, 1, 2048, 3)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)
    text = W.barrier_ladder_text(S0, barrier=0.75, n_spreads=5)
    a = mc.payoffs(il_text.parse(text, ["T"]), mk, {"T": 7}, 0, 1, 2048, 4)
    b = mc.payoffs(cl.compile_contr(C.daily_barrier_cl(S0, barrier=0.75, n_spreads=5)), mk,
                   {"T": 7}, 0, 1, 2048, 4)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)
    assert np.count_nonzero(a == 0.0) > 0 and np.count_nonzero(a) > 0
