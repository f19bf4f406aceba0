"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only *describes* inputs: market parameters, date grids, payoff
programs in the textual IL form, template parameters and seeds.  It holds no
step of the pricing method (no random normals, no path construction, no
payoff evaluation) and imports neither the product package nor the oracle.

The contracts stand in for the paper's OTC workloads (Sec. 6.2, Table 1:
a vanilla European call, a discrete barrier on three underlyings, a double
European on two) and for the benchmark configurations:

* ``european``      -- vanilla call, 1 underlying, 1 observation date;
* ``autocall``      -- worst-of autocallable note on 3 correlated
                       underlyings, 5 annual dates, early redemption at 100%
                       and a knock-in at 60% observed on the annual dates;
* ``daily_barrier`` -- 3 underlyings, 365 daily dates, down-and-out at 70%
                       checked every date, maturity payoff a ladder of call
                       spreads on the worst-of (about 430 IL nodes);
* small contracts for closed-form checks (digital, zero-coupon, forward,
  exchange option) and the portfolio templates.

Every program text is exactly what the CL-to-IL compiler of Sec. 4 produces
for the corresponding CL contract (checked by the oracle tests).  Parties:
0 pays, 1 receives; payoffs are valued from 0 to 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

PARAM_SEED = 0xC0FFEE          # seed of the parameter draws
PATH_SEED_BASE = 0x5EED0001    # path seed of workload k is PATH_SEED_BASE + k

P_PAY, P_RECV = 0, 1


@dataclass
class MarketSpec:
    S0: List[float]
    sigma: List[float]
    corr: List[List[float]]
    r: float
    days: List[int]
    now: int = 0
    history: List[List[float]] = field(default_factory=list)
    hist_days: List[int] = field(default_factory=list)

    @property
    def d(self) -> int:
        return len(self.S0)

    @property
    def n(self) -> int:
        return len(self.days)


@dataclass
class Workload:
    name: str
    market: MarketSpec
    il_text: str
    tparams: List[int]
    n_paths: int
    seed: int
    notional: float            # scale of the per-path tolerance floor
    note: str = ""


def _fmt(x: float) -> str:
    r = repr(float(x))
    return r if any(c in r for c in ".eE") else r + ".0"


def const_corr(d: int, rho: float) -> List[List[float]]:
    return [[1.0 if i == j else rho for j in range(d)] for i in range(d)]


def draw_sigmas(d: int, lo: float = 0.15, hi: float = 0.35, seed: int = PARAM_SEED) -> List[float]:
    """sigma_i ~ U(lo, hi) from a Mersenne-Twister stream."""
    g = np.random.Generator(np.random.MT19937(seed))
    return [float(v) for v in g.uniform(lo, hi, size=d)]


# ---------------------------------------------------------------------------
# Program texts (compiled form of the CL contracts)
# ---------------------------------------------------------------------------


def european_text(K: float) -> str:
    """translate($0, scale(max(obs(0,0) - K, 0), transfer(0,1)))."""
    T = "(tplus 0 $0)"
    return (f"(mult (max (sub (model 0 (tplus {T} 0)) {_fmt(K)}) 0.0) "
            f"(payoff {T} {P_PAY} {P_RECV}))")


def european_if_text(K: float) -> str:
    """The paper's Example 1 shape: translate($0, if(obs(0,0) > K,
    scale(obs(0,0) - K, transfer(0,1)), zero))."""
    T = "(tplus 0 $0)"
    m = f"(model 0 (tplus {T} 0))"
    return (f"(loopif (lt {_fmt(K)} {m}) (mult (sub {m} {_fmt(K)}) "
            f"(payoff {T} {P_PAY} {P_RECV})) 0.0 0)")


def digital_text(K: float) -> str:
    """translate($0, scale(cond(obs(0,0) > K, 1, 0), transfer(0,1)))."""
    T = "(tplus 0 $0)"
    m = f"(model 0 (tplus {T} 0))"
    return f"(mult (if (lt {_fmt(K)} {m}) 1.0 0.0) (payoff {T} {P_PAY} {P_RECV}))"


def zero_coupon_text() -> str:
    """translate($0, transfer(0,1))."""
    return f"(payoff (tplus 0 $0) {P_PAY} {P_RECV})"


def forward_text(K: float) -> str:
    """translate($0, scale(obs(0,0) - K, transfer(0,1)))."""
    T = "(tplus 0 $0)"
    return f"(mult (sub (model 0 (tplus {T} 0)) {_fmt(K)}) (payoff {T} {P_PAY} {P_RECV}))"


def exchange_text() -> str:
    """translate($0, scale(max(obs(0,0) - obs(1,0), 0), transfer(0,1)))."""
    T = "(tplus 0 $0)"
    return (f"(mult (max (sub (model 0 (tplus {T} 0)) (model 1 (tplus {T} 0))) 0.0) "
            f"(payoff {T} {P_PAY} {P_RECV}))")


def worst_text(d: int, S0: Sequence[float], t: str) -> str:
    """min over i of obs(i, .) / S0_i, left-nested."""
    terms = [f"(div (model {i} {t}) {_fmt(S0[i])})" for i in range(d)]
    out = terms[0]
    for x in terms[1:]:
        out = f"(min {out} {x})"
    return out


def autocall_text(S0: Sequence[float], n_dates: int = 5, coupon: float = 0.05,
                  call_level: float = 1.0, ki_level: float = 0.6) -> str:
    """Worst-of autocallable (compiled form of ``autocall_cl`` in the oracle's
    test contracts): on annual date k < n, if worst >= call_level pay
    1 + coupon*k at k, else continue; at date n pay 1 + coupon*n if called,
    else worst if any annual worst <= ki_level (knock-in), else 1."""
    d = len(S0)

    def W(k: int) -> str:
        return worst_text(d, S0, str(k))

    def pay(k: int) -> str:
        return f"(payoff {k} {P_PAY} {P_RECV})"

    n = n_dates
    # or(le(W(0)), or(le(W(-1)), ... )) at maturity, right-nested
    kis = [f"(le {W(n - j)} {_fmt(ki_level)})" for j in range(n)]
    ki = kis[-1]
    for x in reversed(kis[:-1]):
        ki = f"(or {x} {ki})"
    maturity_else = f"(mult (if {ki} {W(n)} 1.0) {pay(n)})"
    body = (f"(loopif (le {_fmt(call_level)} {W(n)}) "
            f"(mult {_fmt(1.0 + coupon * n)} {pay(n)}) {maturity_else} 0)")
    for k in range(n - 1, 0, -1):
        body = (f"(loopif (le {_fmt(call_level)} {W(k)}) "
                f"(mult {_fmt(1.0 + coupon * k)} {pay(k)}) {body} 0)")
    return body


def barrier_ladder_text(S0: Sequence[float], barrier: float = 0.7,
                        n_spreads: int = 13, top: float = 1.95) -> str:
    """Daily down-and-out on the worst-of (compiled form of
    ``daily_barrier_cl``): loopif over $0 days testing any S_i/S0_i <= barrier;
    knocked out pays 0, otherwise at day $0 a ladder of call spreads on the
    worst-of, sum_k (max(W - a_k, 0) - max(W - a_{k+1}, 0)),
    a_k = k * top / n_spreads."""
    d = len(S0)
    hits = [f"(le (div (model {i} 0) {_fmt(S0[i])}) {_fmt(barrier)})" for i in range(d)]
    hit = hits[0]
    for x in hits[1:]:
        hit = f"(or {hit} {x})"
    W = worst_text(d, S0, "0")
    a = [k * top / n_spreads for k in range(n_spreads + 1)]
    terms = [f"(sub (max (sub {W} {_fmt(a[k])}) 0.0) (max (sub {W} {_fmt(a[k + 1])}) 0.0))"
             for k in range(n_spreads)]
    ladder = terms[0]
    for x in terms[1:]:
        ladder = f"(add {ladder} {x})"
    return f"(loopif {hit} 0.0 (mult {ladder} (payoff 0 {P_PAY} {P_RECV})) $0)"


# ---------------------------------------------------------------------------
# Benchmark / parity workloads
# ---------------------------------------------------------------------------


def european_call(n_paths: int = 1 << 16) -> Workload:
    """S0 = K = 100, r = 0.03, sigma = 0.2, T = 1y (one date at day 365)."""
    mk = MarketSpec([100.0], [0.2], [[1.0]], 0.03, [365])
    return Workload("european_call_1u_1d", mk, european_text(100.0), [1], n_paths,
                    PATH_SEED_BASE + 0, 100.0)


def worst_of_autocall(n_paths: int = 1 << 20) -> Workload:
    """3 correlated GBMs, S0 = 1, sigma ~ U(0.15, 0.35), pairwise corr 0.5,
    r = 0.03, annual dates over 5 years."""
    d = 3
    mk = MarketSpec([1.0] * d, draw_sigmas(d), const_corr(d, 0.5), 0.03,
                    [365 * k for k in range(1, 6)])
    return Workload("worst_of_autocall_3u_5d", mk, autocall_text(mk.S0), [], n_paths,
                    PATH_SEED_BASE + 1, 1.0)


def daily_barrier(n_paths: int = 1 << 22) -> Workload:
    """3 correlated GBMs as the autocall, 365 daily dates, barrier 70%."""
    d = 3
    mk = MarketSpec([1.0] * d, draw_sigmas(d), const_corr(d, 0.5), 0.03,
                    list(range(1, 366)))
    return Workload("daily_barrier_3u_365d", mk, barrier_ladder_text(mk.S0), [365],
                    n_paths, PATH_SEED_BASE + 2, 1.0)


def reverse_asian_text(n: int, K: float = 1.0) -> str:
    """Average of assets 0 and 1 over the n dates ending at $0, summed newest
    fixing first (each term looks one date further back): a program that
    is not streamable in a short window (lookback n - 1)."""
    T = "(tplus 0 $0)"
    terms = [f"(add (model 0 (tplus {T} {-j})) (model 1 (tplus {T} {-j})))" for j in range(n)]
    s = terms[0]
    for x in terms[1:]:
        s = f"(add {s} {x})"
    return f"(mult (max (sub (div {s} {float(2 * n)}) {_fmt(K)}) 0.0) (payoff {T} 0 1))"


def reverse_asian(n_paths: int = 1 << 20) -> Workload:
    """2 correlated GBMs (corr 0.5), 300 daily dates, the average-rate call
    summed newest fixing first: window of 512 dates, kept in HBM."""
    d = 2
    mk = MarketSpec([1.0] * d, draw_sigmas(d), const_corr(d, 0.5), 0.03, list(range(1, 301)))
    return Workload("reverse_asian_2u_300d", mk, reverse_asian_text(300), [300], n_paths,
                    PATH_SEED_BASE + 3, 1.0)


def basket_call_greeks(n_paths: int = 1 << 20) -> Workload:
    """The autocall's market (3 GBMs, 5 annual dates) with an equally
    weighted basket call struck at 1 paid at the fifth date: Lipschitz in
    the path, so pathwise delta and vega hold."""
    mk = worst_of_autocall().market
    return Workload("greeks_basket_call_3u_5d", mk, basket_call_text(3, 1.0), [5], n_paths,
                    PATH_SEED_BASE + 4, 1.0)


def daily_barrier_greeks(n_paths: int = 1 << 20) -> Workload:
    """The daily barrier contract on four correlated GBMs (S0 = 1, sigma
    drawn as above, pairwise corr 0.5, 365 daily dates): delta and vega of
    four underlyings, the knock-out decisions held fixed."""
    d = 4
    mk = MarketSpec([1.0] * d, draw_sigmas(d), const_corr(d, 0.5), 0.03, list(range(1, 366)))
    return Workload("greeks_daily_barrier_4u_365d", mk, barrier_ladder_text(mk.S0), [365], n_paths,
                    PATH_SEED_BASE + 5, 1.0)


ALL = {
    "european_call_1u_1d": european_call,
    "worst_of_autocall_3u_5d": worst_of_autocall,
    "daily_barrier_3u_365d": daily_barrier,
    "reverse_asian_2u_300d": reverse_asian,
}
GREEKS = {"greeks_basket_call_3u_5d": basket_call_greeks,
          "greeks_daily_barrier_4u_365d": daily_barrier_greeks}


# ---------------------------------------------------------------------------
# Portfolio of templated contracts (batched pricing)
# ---------------------------------------------------------------------------


def basket_text(d: int, t: str) -> str:
    """(S_0 + ... + S_{d-1}) / d at time t (every S0 = 1), left-nested."""
    out = f"(model 0 {t})"
    for i in range(1, d):
        out = f"(add {out} (model {i} {t}))"
    return f"(div {out} {_fmt(float(d))})"


def basket_call_text(d: int, K: float) -> str:
    """translate($0, scale(max(basket - K, 0), transfer))."""
    T = "(tplus 0 $0)"
    return (f"(mult (max (sub {basket_text(d, f'(tplus {T} 0)')} {_fmt(K)}) 0.0) "
            f"(payoff {T} {P_PAY} {P_RECV}))")


def basket_digital_text(d: int, K: float) -> str:
    """translate($0, scale(cond(basket > K, 1, 0), transfer))."""
    T = "(tplus 0 $0)"
    return (f"(mult (if (lt {_fmt(K)} {basket_text(d, f'(tplus {T} 0)')}) 1.0 0.0) "
            f"(payoff {T} {P_PAY} {P_RECV}))")


def call_spread_text(d: int, K1: float, K2: float) -> str:
    """translate($0, scale(max(basket - K1, 0) - max(basket - K2, 0), transfer))."""
    T = "(tplus 0 $0)"
    b = basket_text(d, f"(tplus {T} 0)")
    return (f"(mult (sub (max (sub {b} {_fmt(K1)}) 0.0) (max (sub {b} {_fmt(K2)}) 0.0)) "
            f"(payoff {T} {P_PAY} {P_RECV}))")


def asian_text(n: int, S0: float, K: float) -> str:
    """translate($0, scale(max((sum_{j<n} obs(0,-j)) / n / S0 - K, 0), transfer)):
    average-rate call on the n grid dates ending at maturity $0 = n.  The
    sum runs in date order (oldest fixing first), so each fixing is read as
    it is simulated."""
    T = "(tplus 0 $0)"
    terms = [f"(model 0 (tplus {T} {-j}))" for j in reversed(range(n))]
    s = terms[0]
    for x in terms[1:]:
        s = f"(add {s} {x})"
    return (f"(mult (max (sub (div (div {s} {_fmt(float(n))}) {_fmt(S0)}) {_fmt(K)}) 0.0) "
            f"(payoff {T} {P_PAY} {P_RECV}))")


@dataclass
class PortfolioItem:
    template: str
    market: MarketSpec
    il_text: str
    tparams: List[int]
    n_paths: int
    notional: float


PORTFOLIO_TEMPLATES = ("european", "digital", "call_spread", "autocall", "daily_barrier", "asian")


def portfolio(n_contracts: int = 1024, seed: int = PARAM_SEED + 4) -> List[PortfolioItem]:
    """Templated contracts on one 4-asset market (S0 = 1, sigma as the
    autocall's draws plus one more, pairwise corr 0.5, r = 3 %): each
    contract draws a template, d ~ U{1..4} underlyings (the first d assets;
    the European, digital and call-spread pay on their equally weighted
    basket, the average-rate call on the first asset),
    a maturity ~ U(0.5, 10) years, a date count ~ log-U{1..365} (evenly
    spaced to maturity), a strike level ~ U(0.8, 1.2) and a path budget
    ~ lognormal clipped to [2^12, 2^18]."""
    g = np.random.Generator(np.random.MT19937(seed))
    sig4 = draw_sigmas(4)
    items = []
    for c in range(n_contracts):
        tmpl = PORTFOLIO_TEMPLATES[int(g.integers(len(PORTFOLIO_TEMPLATES)))]
        d = int(g.integers(1, 5))
        years = float(g.uniform(0.5, 10.0))
        n = int(np.clip(np.round(np.exp(g.uniform(0.0, np.log(365.0)))), 1, 365))
        if tmpl == "asian":
            n = min(n, 200)
        last = max(int(round(years * 365)), n)
        days = sorted({max(1, int(round(last * (k + 1) / n))) for k in range(n)})
        n = len(days)
        strike = float(g.uniform(0.8, 1.2))
        budget = int(np.clip(np.exp(g.normal(np.log(2.0 ** 15), 1.0)), 2 ** 12, 2 ** 18))
        S0 = [1.0] * d
        mk = MarketSpec(S0, sig4[:d], const_corr(d, 0.5), 0.03, days)
        if tmpl == "european":
            text, tp = basket_call_text(d, strike), [n]
        elif tmpl == "digital":
            text, tp = basket_digital_text(d, strike), [n]
        elif tmpl == "call_spread":
            text, tp = call_spread_text(d, strike, strike + 0.2), [n]
        elif tmpl == "autocall":
            text, tp = autocall_text(S0, n_dates=min(n, 12)), []
            mk = MarketSpec(S0, sig4[:d], const_corr(d, 0.5), 0.03, days[:min(n, 12)])
        elif tmpl == "daily_barrier":
            text, tp = barrier_ladder_text(S0, barrier=0.6 + 0.1 * strike, n_spreads=1 + c % 13), [n]
        else:
            text, tp = asian_text(n, 1.0, strike), [n]
        items.append(PortfolioItem(tmpl, mk, text, tp, budget, 1.0))
    return items
