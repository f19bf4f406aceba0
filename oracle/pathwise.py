"""Pathwise sensitivities of the per-path payoff (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For each path, the payoff of Fig. 3 on the simulated environment is a
function of the market parameters S0_l and sigma_l through the GBM map of
``paths`` (the normals stay fixed: common random numbers).  The average
over paths of its derivative estimates d price / d S0_l (delta) and
d price / d sigma_l (vega) for payoffs that are Lipschitz in the path.
Two independent computations of the per-path derivative:

* ``pathwise``: from its definition, a central difference of the oracle's
  own FP64 per-path payoff with a small relative step; away from the points
  where a discrete decision (a comparison) changes, the pathwise derivative
  to about 1e-9 relative.
* ``adjoint``: the chain rule, in reverse.  The IL expression is evaluated
  as in Fig. 3 (each path takes its own branches and loop exits), and the
  derivative of the result with respect to every value it was computed from
  flows back through the arithmetic with the decisions held fixed: add and
  sub pass it on (with sign), mult and div by the partial derivatives, max
  and min to the operand they chose, if and loopif to the branch the path
  took; comparisons, booleans, nats, literals and payoff discounts take
  none.  A model read of label l at ordinal o receives the derivative
  dx/dS_l(o); under GBM, S_l(o) = S0_l exp((r - sigma_l^2/2) tau_o +
  sigma_l X_l(o)) with X = L W independent of the parameters, so
  dS_l(o)/dS0_l = S_l(o) / S0_l and dS_l(o)/dsigma_l = S_l(o) (X_l(o) -
  sigma_l tau_o) (the spot, ordinal 0, has 1 and 0; history has none).
  Every underlying's delta and vega come from one reverse pass.
"""
from __future__ import annotations

import copy
from typing import Mapping, Tuple

import numpy as np

from . import il as IL
from .mc import payoffs
from .paths import Market, simulate_sx


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


def adjoint(il: IL.IL, mk: Market, delta: Mapping[str, int], p1: int, p2: int, n_paths: int,
            seed: int, stream: int = 0, offset: int = 0) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Per path (paths offset .. offset + n_paths - 1): the payoff x and its
    derivatives dx/dS0[p, l] and dx/dsigma[p, l] for every underlying l, by
    one reverse pass (see the module docstring)."""
    paths = np.arange(offset, offset + n_paths, dtype=np.uint64)
    S, X = simulate_sx(mk, seed, stream, paths)
    tau = mk.tau()
    S0 = np.asarray(mk.S0, dtype=np.float64)
    sig = np.asarray(mk.sigma, dtype=np.float64)
    dS0 = np.zeros((n_paths, mk.d))
    dsig = np.zeros((n_paths, mk.d))

    def rho(label: int, t: int, idx: np.ndarray) -> np.ndarray:
        o = t - mk.now
        if 0 <= o <= mk.n:
            return S[idx, label, o]
        if o < 0 and -o <= len(mk.history):
            return np.full(len(idx), float(mk.history[-o - 1][label]))
        raise IndexError(f"model time {t} (ordinal {o}) outside the grid")

    def read_back(label: int, t: int, idx: np.ndarray):
        o = t - mk.now

        def back(g: np.ndarray) -> None:
            if 1 <= o <= mk.n:
                s = S[idx, label, o]
                dS0[idx, label] += g * s / S0[label]
                dsig[idx, label] += g * s * (X[idx, label, o] - sig[label] * tau[o])
            elif o == 0:
                dS0[idx, label] += g
        return back

    args = IL.Args(rho=rho, delta=delta, now=mk.now, d=mk.disc, p1=p1, p2=p2)
    x, back = _reverse(il, args, 0, np.arange(n_paths), read_back)
    if x.dtype != np.float64:
        raise TypeError("a payoff expression must evaluate to a real")
    back(np.ones(n_paths))
    return x, dS0, dsig


def _noop(g: np.ndarray) -> None:
    pass


def _reverse(il: IL.IL, a: IL.Args, t0: int, idx: np.ndarray, read_back):
    """(value as IL[[il]] of Fig. 3 on the paths idx, back) where back(g)
    adds g times the derivative of the value to the model reads' ledger."""
    if isinstance(il, IL.Model):
        t = IL.tsem(il.t, a.delta) + t0
        return np.asarray(a.rho(il.label, t, idx), dtype=IL.REAL), read_back(il.label, t, idx)
    if isinstance(il, IL.UnOp):
        v, b = _reverse(il.e, a, t0, idx, read_back)
        if il.op == "neg" and v.dtype == IL.REAL:
            return -v, (lambda g: b(-g))
        return IL._unop(il.op, v), _noop
    if isinstance(il, IL.BinOp):
        x, bx = _reverse(il.a, a, t0, idx, read_back)
        y, by = _reverse(il.b, a, t0, idx, read_back)
        v = IL._binop(il.op, x, y)
        if v.dtype != IL.REAL:
            return v, _noop
        op = il.op
        if op == "add":
            return v, (lambda g: (bx(g), by(g)))
        if op == "sub":
            return v, (lambda g: (bx(g), by(-g)))
        if op == "mult":
            return v, (lambda g: (bx(g * y), by(g * x)))
        if op == "div":
            return v, (lambda g: (bx(g / y), by(-g * x / (y * y))))
        if op in ("max", "min"):
            first = x >= y if op == "max" else x <= y
            return v, (lambda g: (bx(np.where(first, g, 0.0)), by(np.where(first, 0.0, g))))
        raise TypeError(f"no derivative rule for {op}")
    if isinstance(il, IL.If):
        c = IL._ev(il.c, a, t0, idx)
        if IL._kind(c) != "bool":
            raise TypeError("if condition must be bool")
        return _merge_rev([(np.nonzero(c)[0], il.a, t0), (np.nonzero(~c)[0], il.b, t0)], a, idx, read_back)
    if isinstance(il, IL.LoopIf):
        n = IL.tsem(il.t, a.delta)
        parts = []
        pending = np.arange(len(idx))
        for k in range(n + 1):
            if len(pending) == 0:
                break
            c = IL._ev(il.c, a, t0 + k, idx[pending])
            if IL._kind(c) != "bool":
                raise TypeError("loopif condition must be bool")
            parts.append((pending[c], il.a, t0 + k))
            pending = pending[~c]
        parts.append((pending, il.b, t0 + n))
        return _merge_rev(parts, a, idx, read_back)
    # literals, time expressions, now, payoff: no derivative
    return IL._ev(il, a, t0, idx), _noop


def _merge_rev(parts, a: IL.Args, idx: np.ndarray, read_back):
    """Branches evaluated on the paths (positions) that took them; the
    derivative of each position flows back into its own branch."""
    out, backs = None, []
    for pos, expr, t0 in parts:
        if len(pos) == 0:
            continue
        v, b = _reverse(expr, a, t0, idx[pos], read_back)
        if out is None:
            out = np.empty(len(idx), dtype=v.dtype)
        elif out.dtype != v.dtype:
            raise TypeError("branches of different types")
        out[pos] = v
        backs.append((pos, b))
    if out is None:
        out = np.empty(0, dtype=IL.REAL)

    def back(g: np.ndarray) -> None:
        for pos, b in backs:
            b(g[pos])
    return out, back
