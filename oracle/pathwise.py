"""Pathwise sensitivities of the per-path payoff (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For each path, the payoff of Fig. 3 on the simulated environment is a
function of the market parameters S0_l and sigma_l through the GBM map of
``paths`` (the normals stay fixed: common random numbers).  Its derivative
is taken here from its definition, as a central difference of the oracle's
own FP64 per-path payoff with a small relative step; away from the points
where a discrete decision (a comparison) changes, this is the pathwise
derivative to about 1e-9 relative.  The average over paths estimates
d price / d S0_l (delta) and d price / d sigma_l (vega) for payoffs that
are Lipschitz in the path.
"""
from __future__ import annotations

import copy
from typing import Mapping, Tuple

import numpy as np

from . import il as IL
from .mc import payoffs
from .paths import Market


def _bumped(mk: Market, field: str, label: int, h: float) -> Market:
    m = copy.deepcopy(mk)
    vals = list(getattr(m, field))
    vals[label] = vals[label] + h
    setattr(m, field, vals)
    return m


def pathwise(il: IL.IL, mk: Market, delta: Mapping[str, int], p1: int, p2: int, n_paths: int,
             seed: int, label: int, stream: int = 0, offset: int = 0,
             rel_step: float = 1e-6) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Per path: (payoff, d payoff / d S0[label], d payoff / d sigma[label],
    tie margin of the unbumped evaluation)."""
    x, marg = payoffs(il, mk, delta, p1, p2, n_paths, seed, stream, offset, with_margins=True)
    out = []
    for field in ("S0", "sigma"):
        h = rel_step * max(abs(getattr(mk, field)[label]), 1e-3)
        up = payoffs(il, _bumped(mk, field, label, h), delta, p1, p2, n_paths, seed, stream, offset)
        dn = payoffs(il, _bumped(mk, field, label, -h), delta, p1, p2, n_paths, seed, stream, offset)
        out.append((up - dn) / (2.0 * h))
    return x, out[0], out[1], marg
