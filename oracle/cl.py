"""Contract language CL: syntax, trace semantics, instantiation, compiler to IL.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Annenkov & Elsman, "Certified Compilation of Financial Contracts":

* syntax ``Contr`` / ``Exp`` / ``TExpr``        -- Fig. 1;
* ``esem`` (E[[e]]) and ``csem`` (C[[c]])       -- Sec. 2 (the semantics of
  Bahr, Berthold & Elsman extended with a template environment; translate
  delays by T[t]delta);
* ``inst``                                      -- Definition 1;
* ``horizon``                                   -- the conservative bound
  HOR_delta(c) used in Theorem 1;
* ``compile_exp`` / ``compile_contr``           -- tau_e / tau_c of Sec. 4.

Readings: transfer(p1, p2, a) gives a unit flow from p1 to p2 at time 0,
recorded as +1 on (p1, p2) and -1 on (p2, p1); assets are dropped (the IL
has a single currency, Sec. 4 compiles transfer to payoff(t0, p1, p2)).
scale(e, c) multiplies every flow of c by the value of e at the time the
scale is reached.  ifWithin(e, t, c1, c2) tests e at offsets 0..T[t]delta
and continues as c1 delayed by the first offset where e holds, else as c2
delayed by T[t]delta.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Dict, Mapping, Tuple, Union

from . import il as IL
from .il import TNum, TVar, TimeExpr, tsem, tplus

# ---------------------------------------------------------------------------
# Syntax (Fig. 1)
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Op:
    """op(e1, ..., en) with op in add sub mult div lt le eq neg not and or
    max min cond."""
    op: str
    args: Tuple["Exp", ...]


@dataclass(frozen=True)
class Obs:
    """obs(l, i): observable l at relative time i (i may be negative)."""
    label: int
    i: int


@dataclass(frozen=True)
class RLit:
    f: float


@dataclass(frozen=True)
class BLit:
    b: bool


Exp = Union[Op, Obs, RLit, BLit]


@dataclass(frozen=True)
class Zero:
    pass


@dataclass(frozen=True)
class Transfer:
    p1: int
    p2: int
    asset: str = "EUR"


@dataclass(frozen=True)
class Scale:
    e: Exp
    c: "Contr"


@dataclass(frozen=True)
class Translate:
    t: TimeExpr
    c: "Contr"


@dataclass(frozen=True)
class IfWithin:
    e: Exp
    t: TimeExpr
    c1: "Contr"
    c2: "Contr"


@dataclass(frozen=True)
class Both:
    c1: "Contr"
    c2: "Contr"


Contr = Union[Zero, Transfer, Scale, Translate, IfWithin, Both]

Env = Callable[[int, int], float]          # rho(label, time) -> value
Trace = Dict[int, Dict[Tuple[int, int], float]]


def shift(rho: Env, k: int) -> Env:
    """rho/k: the environment advanced by k time steps."""
    return lambda l, i: rho(l, i + k)


# ---------------------------------------------------------------------------
# Expression semantics E[[e]]
# ---------------------------------------------------------------------------

_BIN = {
    "add": lambda x, y: x + y,
    "sub": lambda x, y: x - y,
    "mult": lambda x, y: x * y,
    "div": lambda x, y: x / y,
    "lt": lambda x, y: x < y,
    "le": lambda x, y: x <= y,
    "eq": lambda x, y: x == y,
    "max": lambda x, y: max(x, y),
    "min": lambda x, y: min(x, y),
}


def _is_real(v) -> bool:
    return type(v) is float


def _is_bool(v) -> bool:
    return type(v) is bool


def esem(e: Exp, rho: Env):
    """E[[e]]rho: the value (float or bool) of a CL expression at the current
    time of environment rho; observables come from rho(l, i)."""
    if isinstance(e, RLit):
        return float(e.f)
    if isinstance(e, BLit):
        return bool(e.b)
    if isinstance(e, Obs):
        return float(rho(e.label, e.i))
    if isinstance(e, Op):
        vs = [esem(x, rho) for x in e.args]
        if e.op == "cond":
            b, x, y = vs
            if not _is_bool(b):
                raise TypeError("cond on non-bool")
            return x if b else y
        if e.op == "neg":
            (x,) = vs
            if not _is_real(x):
                raise TypeError("neg on non-real")
            return -x
        if e.op == "not":
            (x,) = vs
            if not _is_bool(x):
                raise TypeError("not on non-bool")
            return not x
        if e.op in ("and", "or"):
            x, y = vs
            if not (_is_bool(x) and _is_bool(y)):
                raise TypeError(f"{e.op} on non-bool")
            return (x and y) if e.op == "and" else (x or y)
        if e.op == "eq" and _is_bool(vs[0]) and _is_bool(vs[1]):
            return vs[0] == vs[1]
        x, y = vs
        if not (_is_real(x) and _is_real(y)):
            raise TypeError(f"{e.op} on non-real")
        r = _BIN[e.op](x, y)
        return bool(r) if e.op in ("lt", "le", "eq") else float(r)
    raise TypeError(f"not an expression: {e!r}")


# ---------------------------------------------------------------------------
# Contract semantics C[[c]] (Sec. 2)
# ---------------------------------------------------------------------------


def _add_into(dst: Trace, src: Trace, k: int = 0, scale: float = 1.0) -> None:
    for t, tr in src.items():
        row = dst.setdefault(t + k, {})
        for key, v in tr.items():
            row[key] = row.get(key, 0.0) + scale * v


def csem(c: Contr, rho: Env, delta: Mapping[str, int]) -> Trace:
    """C[[c]]_(rho, delta): the trace of c as a sparse map time -> flows."""
    if isinstance(c, Zero):
        return {}
    if isinstance(c, Transfer):
        if c.p1 == c.p2:
            return {}
        return {0: {(c.p1, c.p2): 1.0, (c.p2, c.p1): -1.0}}
    if isinstance(c, Scale):
        s = esem(c.e, rho)
        if not _is_real(s):
            raise TypeError("scale by non-real")
        out: Trace = {}
        _add_into(out, csem(c.c, rho, delta), 0, s)
        return out
    if isinstance(c, Translate):                 # delay(T[t]delta, C[[c]](rho/T))
        k = tsem(c.t, delta)
        out = {}
        _add_into(out, csem(c.c, shift(rho, k), delta), k)
        return out
    if isinstance(c, Both):
        out = {}
        _add_into(out, csem(c.c1, rho, delta))
        _add_into(out, csem(c.c2, rho, delta))
        return out
    if isinstance(c, IfWithin):
        n = tsem(c.t, delta)
        for k in range(n + 1):
            b = esem(c.e, shift(rho, k))
            if not _is_bool(b):
                raise TypeError("ifWithin condition must be bool")
            if b:
                out = {}
                _add_into(out, csem(c.c1, shift(rho, k), delta), k)
                return out
        out = {}
        _add_into(out, csem(c.c2, shift(rho, n), delta), n)
        return out
    raise TypeError(f"not a contract: {c!r}")


def trace_flow(tr: Trace, t: int, p1: int, p2: int) -> float:
    """tr(t)(p1, p2)."""
    return tr.get(t, {}).get((p1, p2), 0.0)


def horizon(c: Contr, delta: Mapping[str, int]) -> int:
    """HOR_delta(c): a conservative bound on the last time carrying a flow
    (flows of c happen at times 0..HOR)."""
    if isinstance(c, (Zero, Transfer)):
        return 0
    if isinstance(c, Scale):
        return horizon(c.c, delta)
    if isinstance(c, Translate):
        return tsem(c.t, delta) + horizon(c.c, delta)
    if isinstance(c, Both):
        return max(horizon(c.c1, delta), horizon(c.c2, delta))
    if isinstance(c, IfWithin):
        return tsem(c.t, delta) + max(horizon(c.c1, delta), horizon(c.c2, delta))
    raise TypeError(c)


# ---------------------------------------------------------------------------
# Instantiation (Definition 1)
# ---------------------------------------------------------------------------


def inst(c: Contr, delta: Mapping[str, int]) -> Contr:
    """inst(c, delta): replace template expressions by their values."""
    if isinstance(c, (Zero, Transfer)):
        return c
    if isinstance(c, Scale):
        return Scale(c.e, inst(c.c, delta))
    if isinstance(c, Translate):
        return Translate(TNum(tsem(c.t, delta)), inst(c.c, delta))
    if isinstance(c, Both):
        return Both(inst(c.c1, delta), inst(c.c2, delta))
    if isinstance(c, IfWithin):
        return IfWithin(c.e, TNum(tsem(c.t, delta)), inst(c.c1, delta), inst(c.c2, delta))
    raise TypeError(c)


def template_closed(c: Contr) -> bool:
    """TC(c) of Fig. 2: no template variables in translate / ifWithin."""
    if isinstance(c, (Zero, Transfer)):
        return True
    if isinstance(c, Scale):
        return template_closed(c.c)
    if isinstance(c, Translate):
        return isinstance(c.t, TNum) and template_closed(c.c)
    if isinstance(c, Both):
        return template_closed(c.c1) and template_closed(c.c2)
    if isinstance(c, IfWithin):
        return isinstance(c.t, TNum) and template_closed(c.c1) and template_closed(c.c2)
    raise TypeError(c)


# ---------------------------------------------------------------------------
# Compiler tau_e / tau_c (Sec. 4)
# ---------------------------------------------------------------------------

_UN = {"neg", "not"}


def compile_exp(e: Exp, t0: TimeExpr) -> IL.IL:
    """tau_e[[e]]_t0: expressions map operator by operator; cond becomes if;
    obs(l, i) becomes model(l, tplus(t0, i))."""
    if isinstance(e, RLit):
        return IL.Float(float(e.f))
    if isinstance(e, BLit):
        return IL.Bool(bool(e.b))
    if isinstance(e, Obs):
        return IL.Model(e.label, tplus(t0, TNum(e.i)))
    if isinstance(e, Op):
        xs = [compile_exp(x, t0) for x in e.args]
        if e.op == "cond":
            return IL.If(*xs)
        if e.op in _UN:
            return IL.UnOp(e.op, xs[0])
        return IL.BinOp(e.op, xs[0], xs[1])
    raise TypeError(e)


def compile_contr(c: Contr, t0: TimeExpr = TNum(0)) -> IL.IL:
    """tau_c[[c]]_t0: zero -> 0; transfer -> payoff(t0, p1, p2);
    scale -> mult; translate accumulates its shift into t0 with tplus;
    both -> add; ifWithin -> loopif with the window t as its bound."""
    if isinstance(c, Zero):
        return IL.Float(0.0)
    if isinstance(c, Transfer):
        return IL.Payoff(t0, c.p1, c.p2)
    if isinstance(c, Scale):
        return IL.BinOp("mult", compile_exp(c.e, t0), compile_contr(c.c, t0))
    if isinstance(c, Translate):
        return compile_contr(c.c, tplus(t0, c.t))
    if isinstance(c, Both):
        return IL.BinOp("add", compile_contr(c.c1, t0), compile_contr(c.c2, t0))
    if isinstance(c, IfWithin):
        return IL.LoopIf(compile_exp(c.e, t0), compile_contr(c.c1, t0),
                         compile_contr(c.c2, t0), c.t)
    raise TypeError(c)


# Convenience constructors used by the test contracts ----------------------


def op(name: str, *args: Exp) -> Op:
    return Op(name, tuple(args))


def gt(x: Exp, y: Exp) -> Op:
    """x > y, written with the lt of the operator set."""
    return Op("lt", (y, x))


def ge(x: Exp, y: Exp) -> Op:
    return Op("le", (y, x))


def all_of(*cs: Contr) -> Contr:
    """all[c1, ..., cn] = both(c1, both(..., cn)) (Sec. 2, Example 2)."""
    if not cs:
        return Zero()
    out = cs[-1]
    for c in reversed(cs[:-1]):
        out = Both(c, out)
    return out


def if_(e: Exp, c1: Contr, c2: Contr) -> Contr:
    """if(e, c1, c2) = ifWithin(e, 0, c1, c2)."""
    return IfWithin(e, TNum(0), c1, c2)
