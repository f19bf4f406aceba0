"""Monte Carlo driver: per-path payoff values and the mean / standard error.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Each path is one external environment rho (Sec. 2: Env maps (time, label) to
values): history for ordinals < 0, the spot at ordinal 0 and the simulated
GBM path for ordinals 1..n.  The payoff of a path is IL[[il]] evaluated with
t0 = 0, t = now and the model's discount function (Fig. 3; Theorem 1 states
that this is the discounted sum of the contract's cashflows).  The price
estimate is the average over paths (Sec. 3: the engine averages simulated
outcomes) and the standard error is sqrt(sample variance / N).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Mapping

import numpy as np

from . import il as IL
from .paths import Market, simulate


def env_from_paths(mk: Market, S: np.ndarray, base: np.ndarray | None = None):
    """rho(label, t, idx) over simulated paths S[p, i, o]; ``idx`` index the
    rows of S."""
    n = mk.n

    def rho(label: int, t: int, idx: np.ndarray) -> np.ndarray:
        if not 0 <= label < mk.d:
            raise IndexError(f"label {label} outside 0..{mk.d - 1}")
        o = t - mk.now
        if 0 <= o <= n:
            return S[idx, label, o]
        if o < 0 and -o <= len(mk.history):
            return np.full(len(idx), float(mk.history[-o - 1][label]))
        raise IndexError(f"model time {t} (ordinal {o}) outside the grid")

    return rho


def payoffs(il: IL.IL, mk: Market, delta: Mapping[str, int], p1: int, p2: int,
            n_paths: int, seed: int, stream: int = 0, offset: int = 0,
            paths: np.ndarray | None = None, with_margins: bool = False):
    """Discounted payoff of each path (global indices offset..offset+n-1, or
    the explicit ``paths``).  With ``with_margins`` also returns each path's
    smallest relative distance of a real comparison from a tie."""
    if paths is None:
        paths = np.arange(offset, offset + n_paths, dtype=np.uint64)
    S = simulate(mk, seed, stream, paths)
    margins = np.full(len(paths), np.inf) if with_margins else None
    args = IL.Args(rho=env_from_paths(mk, S), delta=delta, now=mk.now,
                   d=mk.disc, p1=p1, p2=p2, margins=margins)
    v = IL.evaluate(il, args, t0=0, idx=np.arange(len(paths)))
    if v.dtype != np.float64:
        raise TypeError("a payoff expression must evaluate to a real")
    return (v, margins) if with_margins else v


@dataclass
class Estimate:
    price: float
    stderr: float
    n: int
    sum: float
    sumsq: float


def estimate(x: np.ndarray) -> Estimate:
    """Mean and standard error of the path values, from sum and sum of
    squares accumulated in path order."""
    n = len(x)
    s = 0.0
    s2 = 0.0
    for v in x.tolist():
        s += v
        s2 += v * v
    mean = s / n
    var = (s2 - n * mean * mean) / (n - 1) if n > 1 else float("nan")
    return Estimate(mean, math.sqrt(max(var, 0.0) / n), n, s, s2)


def price(il: IL.IL, mk: Market, delta: Mapping[str, int], p1: int, p2: int,
          n_paths: int, seed: int, stream: int = 0, offset: int = 0,
          chunk: int = 1 << 15) -> Estimate:
    """Monte Carlo price of ``il`` over n_paths paths."""
    parts = []
    for a in range(offset, offset + n_paths, chunk):
        m = min(chunk, offset + n_paths - a)
        parts.append(payoffs(il, mk, delta, p1, p2, m, seed, stream, a))
    return estimate(np.concatenate(parts))
