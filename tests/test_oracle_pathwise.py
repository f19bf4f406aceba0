"""Pins of the oracle's pathwise sensitivities: the averages of the per-path
derivatives match the Black-Scholes delta and vega of a European call
(closed forms), a forward's delta is exactly 1 in expectation and its vega 0
path by path, and a contract on another underlying has zero sensitivity."""
import math

import numpy as np
import pytest

from oracle import cl, closed_forms as cf, contracts as C, pathwise
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
