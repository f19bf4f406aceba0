"""Pins of the oracle's pathwise sensitivities: the averages of the per-path
derivatives match the Black-Scholes delta and vega of a European call
(closed forms), a forward's delta is exactly 1 in expectation and its vega 0
path by path, and a contract on another underlying has zero sensitivity."""
import math

import numpy as np
import pytest

from oracle import cl, closed_forms as cf, contracts as C, il_text, pathwise
from oracle.paths import Market


def within(x, want, k=3.0):
    m, se = x.mean(), x.std(ddof=1) / math.sqrt(len(x))
    assert abs(m - want) <= k * se + 1e-12, (m, want, se)


def test_european_call_delta_vega_against_black_scholes():
    mk = Market([100.0], [0.2], [[1.0]], 0.03, [365])
    prog = cl.compile_contr(C.european_cl(100.0))
    x, dS, dv, _ = pathwise.pathwise(prog, mk, {"T": 1}, 0, 1, 1 << 16, 11, label=0)
    within(dS, cf.bs_delta_call(100, 100, 0.03, 0.2, 1.0))
    within(dv, cf.bs_vega(100, 100, 0.03, 0.2, 1.0))
    # pathwise delta of a call is (S_T / S0) disc on paths in the money
    in_money = x > 0
    np.testing.assert_allclose(dS[~in_money], 0.0, atol=1e-9)


def test_forward_delta_and_vega():
    mk = Market([100.0, 50.0], [0.25, 0.4], [[1, 0.3], [0.3, 1]], 0.02, [90, 365])
    prog = cl.compile_contr(C.forward_cl(100.0))
    x, dS, dv, _ = pathwise.pathwise(prog, mk, {"T": 2}, 0, 1, 1 << 15, 3, label=0)
    # d/dS0 of (S_T - K) disc is S_T / S0 disc, whose mean is exactly 1
    np.testing.assert_allclose(dS, (x + 100.0 * mk.disc(2)) / 100.0, rtol=1e-7)
    within(dS, 1.0)
    within(dv, 0.0)
    # nothing depends on the second underlying
    _, dS1, dv1, _ = pathwise.pathwise(prog, mk, {"T": 2}, 0, 1, 4096, 3, label=1)
    assert np.all(dS1 == 0.0) and np.all(dv1 == 0.0)


def test_exchange_option_delta_against_margrabe():
    mk = Market([100.0, 95.0], [0.25, 0.3], [[1, 0.5], [0.5, 1]], 0.03, [182, 365])
    prog = cl.compile_contr(C.exchange_cl())
    _, dS, _, _ = pathwise.pathwise(prog, mk, {"T": 2}, 0, 1, 1 << 16, 21, label=0)
    s = math.sqrt(0.25 ** 2 + 0.3 ** 2 - 2 * 0.5 * 0.25 * 0.3)
    d1 = (math.log(100.0 / 95.0) + 0.5 * s * s) / s
    within(dS, cf.Phi(d1))


# ---------------------------------------------------------------------------
# The reverse-mode adjoint (oracle.pathwise.adjoint), pinned against closed
# forms and against the central differences of the per-path payoff
# ---------------------------------------------------------------------------


def test_adjoint_european_call_against_black_scholes():
    mk = Market([100.0], [0.2], [[1.0]], 0.03, [365])
    prog = cl.compile_contr(C.european_cl(100.0))
    x, dS, dv = pathwise.adjoint(prog, mk, {"T": 1}, 0, 1, 1 << 16, 11)
    within(dS[:, 0], cf.bs_delta_call(100, 100, 0.03, 0.2, 1.0))
    within(dv[:, 0], cf.bs_vega(100, 100, 0.03, 0.2, 1.0))
    # in the money: d/dS0 = (S_T / S0) disc exactly (x = (S_T - K) disc)
    itm = x > 0
    np.testing.assert_allclose(dS[itm, 0], (x[itm] + 100.0 * mk.disc(1)) / 100.0, rtol=1e-12)
    np.testing.assert_array_equal(dS[~itm, 0], 0.0)


def test_adjoint_exchange_option_against_margrabe():
    """Both underlyings from one pass: Margrabe's exchange option value
    S1 Phi(d1) - S2 Phi(d2) has delta Phi(d1) in S1 and -Phi(d2) in S2."""
    mk = Market([100.0, 95.0], [0.25, 0.3], [[1, 0.5], [0.5, 1]], 0.03, [182, 365])
    prog = cl.compile_contr(C.exchange_cl())
    _, dS, _ = pathwise.adjoint(prog, mk, {"T": 2}, 0, 1, 1 << 16, 21)
    s = math.sqrt(0.25 ** 2 + 0.3 ** 2 - 2 * 0.5 * 0.25 * 0.3)
    d1 = (math.log(100.0 / 95.0) + 0.5 * s * s) / s
    within(dS[:, 0], cf.Phi(d1))
    within(dS[:, 1], -cf.Phi(d1 - s))


def test_adjoint_forward_is_exact():
    """(S_T - K) disc: d/dS0 = S_T / S0 disc and d/dsigma = S_T (X_T -
    sigma T) disc on every path; nothing depends on the second underlying."""
    mk = Market([100.0, 50.0], [0.25, 0.4], [[1, 0.3], [0.3, 1]], 0.02, [90, 365])
    prog = cl.compile_contr(C.forward_cl(100.0))
    x, dS, dv = pathwise.adjoint(prog, mk, {"T": 2}, 0, 1, 4096, 3)
    ST = x + 100.0 * mk.disc(2)
    np.testing.assert_allclose(dS[:, 0], ST / 100.0, rtol=1e-12)
    within(dS[:, 0], 1.0)
    within(dv[:, 0], 0.0)
    assert np.all(dS[:, 1] == 0.0) and np.all(dv[:, 1] == 0.0)


@pytest.mark.parametrize("name", ["european", "forward", "exchange", "autocall", "autocall_scaled",
                                  "worst_knockout", "basket_and", "lookback", "nested_loops",
                                  "double_barrier"])
def test_adjoint_matches_central_differences(name):
    """Per path and per underlying, the chain rule in reverse equals the
    central difference of the oracle's payoff, on paths whose decisions are
    not within 1e-5 of a tie (where the difference straddles a kink)."""
    from cases import CASES
    text, tp, spec, _ = CASES[name]
    prog = il_text.parse(text)
    mk, env = Market(**vars(spec)), {f"${i}": v for i, v in enumerate(tp)}
    n, seed = 512, 0x4242 + len(name)
    x, dS, dv = pathwise.adjoint(prog, mk, env, 0, 1, n, seed)
    for l in range(spec.d):
        fx, fS, fv, marg = pathwise.pathwise(prog, mk, env, 0, 1, n, seed, l)
        np.testing.assert_array_equal(x, fx)
        ok = marg >= 1e-5
        assert ok.mean() > 0.9
        for got, ref, h in ((dS[:, l], fS, 1e-6 * mk.S0[l]), (dv[:, l], fv, 1e-6 * mk.sigma[l])):
            # central differences err by O(h^2) in the curvature and by the
            # payoff's rounding over 2h
            tol = 1e-5 * (np.abs(ref) + np.abs(ref).mean()) + 1e-7 * np.abs(x).max() / h
            assert np.all(np.abs(got - ref)[ok] <= tol[ok]), (name, l, np.max(np.abs(got - ref)[ok]))
