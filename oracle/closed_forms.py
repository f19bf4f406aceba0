"""Closed-form prices used to pin the Monte Carlo oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Textbook Black-Scholes results for a lognormal underlying with constant rate
r and volatility sigma (Black & Scholes 1973; Margrabe 1978 for the exchange
option).  Phi is the standard normal CDF, written with math.erf.
"""
from __future__ import annotations

import math


def Phi(x: float) -> float:
    return 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))


def _d12(S0, K, r, sigma, T):
    d1 = (math.log(S0 / K) + (r + 0.5 * sigma * sigma) * T) / (sigma * math.sqrt(T))
    return d1, d1 - sigma * math.sqrt(T)


def bs_call(S0: float, K: float, r: float, sigma: float, T: float) -> float:
    d1, d2 = _d12(S0, K, r, sigma, T)
    return S0 * Phi(d1) - K * math.exp(-r * T) * Phi(d2)


def bs_put(S0: float, K: float, r: float, sigma: float, T: float) -> float:
    d1, d2 = _d12(S0, K, r, sigma, T)
    return K * math.exp(-r * T) * Phi(-d2) - S0 * Phi(-d1)


def digital_call(S0: float, K: float, r: float, sigma: float, T: float) -> float:
    """Cash-or-nothing: pays 1 at T if S_T > K."""
    _, d2 = _d12(S0, K, r, sigma, T)
    return math.exp(-r * T) * Phi(d2)


def zero_coupon(r: float, T: float) -> float:
    return math.exp(-r * T)


def forward(S0: float, K: float, r: float, T: float) -> float:
    """Value of receiving S_T - K at T."""
    return S0 - K * math.exp(-r * T)


def margrabe(S1: float, S2: float, s1: float, s2: float, rho: float, T: float) -> float:
    """Option to exchange asset 2 for asset 1: pays max(S1_T - S2_T, 0)."""
    s = math.sqrt(s1 * s1 + s2 * s2 - 2.0 * rho * s1 * s2)
    d1 = (math.log(S1 / S2) + 0.5 * s * s * T) / (s * math.sqrt(T))
    return S1 * Phi(d1) - S2 * Phi(d1 - s * math.sqrt(T))


def bs_delta_call(S0: float, K: float, r: float, sigma: float, T: float) -> float:
    d1, _ = _d12(S0, K, r, sigma, T)
    return Phi(d1)


def bs_vega(S0: float, K: float, r: float, sigma: float, T: float) -> float:
    d1, _ = _d12(S0, K, r, sigma, T)
    return S0 * math.exp(-0.5 * d1 * d1) / math.sqrt(2.0 * math.pi) * math.sqrt(T)
