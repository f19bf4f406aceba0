"""CL definitions of the test and benchmark contracts.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

These are the contracts of the synthetic workloads written in the contract
language of Fig. 1; ``cl.compile_contr`` (Sec. 4) turns each into the payoff
expression the engine prices.  Parties: 0 pays, 1 receives.  Template
variable ``T`` (printed ``$0``) is a maturity or window in date ordinals.
"""
from __future__ import annotations

from typing import Sequence

from .cl import (BLit, Both, IfWithin, Obs, Op, RLit, Scale, Transfer, Translate,
                 Zero, ge, gt, if_, op)
from .il import TNum, TVar

PAY, RECV = 0, 1
T = TVar("T")


def xfer() -> Transfer:
    return Transfer(PAY, RECV)


def european_cl(K: float) -> Scale:
    """translate(T, scale(max(obs(0,0) - K, 0), transfer))."""
    return Translate(T, Scale(op("max", op("sub", Obs(0, 0), RLit(K)), RLit(0.0)), xfer()))


def european_if_cl(K: float):
    """The templated call of Sec. 2: translate(T, if(obs > K,
    scale(obs - K, transfer), zero))."""
    return Translate(T, if_(gt(Obs(0, 0), RLit(K)),
                            Scale(op("sub", Obs(0, 0), RLit(K)), xfer()), Zero()))


def digital_cl(K: float):
    return Translate(T, Scale(op("cond", gt(Obs(0, 0), RLit(K)), RLit(1.0), RLit(0.0)), xfer()))


def zero_coupon_cl():
    return Translate(T, xfer())


def forward_cl(K: float):
    return Translate(T, Scale(op("sub", Obs(0, 0), RLit(K)), xfer()))


def exchange_cl():
    return Translate(T, Scale(op("max", op("sub", Obs(0, 0), Obs(1, 0)), RLit(0.0)), xfer()))


def worst(S0: Sequence[float], i: int):
    """min_k obs(k, i) / S0_k, left-nested."""
    out = op("div", Obs(0, i), RLit(S0[0]))
    for k in range(1, len(S0)):
        out = op("min", out, op("div", Obs(k, i), RLit(S0[k])))
    return out


def autocall_cl(S0: Sequence[float], n_dates: int = 5, coupon: float = 0.05,
                call_level: float = 1.0, ki_level: float = 0.6):
    """Worst-of autocallable: a chain of one-date ifWithin's, one year apart.
    Called at date k (worst >= call_level): pay 1 + coupon*k.  Not called by
    date n: pay worst if any annual worst was <= ki_level, else 1; the
    knock-in looks back with obs(., -j)."""
    n = n_dates
    kis = [op("le", worst(S0, -j), RLit(ki_level)) for j in range(n)]
    ki = kis[-1]
    for x in reversed(kis[:-1]):
        ki = op("or", x, ki)
    last = if_(ge(worst(S0, 0), RLit(call_level)),
               Scale(RLit(1.0 + coupon * n), xfer()),
               Scale(op("cond", ki, worst(S0, 0), RLit(1.0)), xfer()))
    body = last
    for k in range(n - 1, 0, -1):
        body = if_(ge(worst(S0, 0), RLit(call_level)),
                   Scale(RLit(1.0 + coupon * k), xfer()),
                   Translate(TNum(1), body))
    return Translate(TNum(1), body)


def daily_barrier_cl(S0: Sequence[float], barrier: float = 0.7,
                     n_spreads: int = 13, top: float = 1.95):
    """ifWithin(any S_i/S0_i <= barrier, T, zero, scale(ladder, transfer)):
    knocked out on the first day the barrier is touched, otherwise at day T
    the ladder of call spreads on the worst-of."""
    hit = op("le", op("div", Obs(0, 0), RLit(S0[0])), RLit(barrier))
    for k in range(1, len(S0)):
        hit = op("or", hit, op("le", op("div", Obs(k, 0), RLit(S0[k])), RLit(barrier)))
    W = worst(S0, 0)
    a = [k * top / n_spreads for k in range(n_spreads + 1)]
    terms = [op("sub", op("max", op("sub", W, RLit(a[k])), RLit(0.0)),
                op("max", op("sub", W, RLit(a[k + 1])), RLit(0.0)))
             for k in range(n_spreads)]
    ladder = terms[0]
    for x in terms[1:]:
        ladder = op("add", ladder, x)
    return IfWithin(hit, T, Zero(), Scale(ladder, xfer()))


def basket(d: int):
    """(obs(0,0) + ... + obs(d-1,0)) / d, left-nested (every S0 = 1)."""
    s = Obs(0, 0)
    for i in range(1, d):
        s = op("add", s, Obs(i, 0))
    return op("div", s, RLit(float(d)))


def basket_call_cl(d: int, K: float):
    """translate(T, scale(max(basket - K, 0), transfer))."""
    return Translate(T, Scale(op("max", op("sub", basket(d), RLit(K)), RLit(0.0)), xfer()))


def basket_digital_cl(d: int, K: float):
    return Translate(T, Scale(op("cond", gt(basket(d), RLit(K)), RLit(1.0), RLit(0.0)), xfer()))


def call_spread_cl(d: int, K1: float, K2: float):
    """translate(T, scale(max(basket - K1, 0) - max(basket - K2, 0), transfer))."""
    return Translate(T, Scale(op("sub", op("max", op("sub", basket(d), RLit(K1)), RLit(0.0)),
                                 op("max", op("sub", basket(d), RLit(K2)), RLit(0.0))), xfer()))


def asian_cl(n: int, S0: float, K: float):
    """Average-rate call: translate(T, scale(max(mean_{j<n} obs(0,-j) / S0 - K, 0),
    transfer)), the mean over the n grid dates ending at T, summed oldest
    fixing first."""
    s = Obs(0, -(n - 1))
    for j in reversed(range(n - 1)):
        s = op("add", s, Obs(0, -j))
    avg = op("div", op("div", s, RLit(float(n))), RLit(S0))
    return Translate(T, Scale(op("max", op("sub", avg, RLit(K)), RLit(0.0)), xfer()))
