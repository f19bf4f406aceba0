"""Payoff intermediate language (IL): syntax, semantics, compiler, cutPayoff.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Annenkov & Elsman, "Certified Compilation of Financial Contracts":

* syntax            -- Sec. 3 grammar and the Coq ``ILExpr`` / ``ILTExprZ``
                       definitions of Sec. 5;
* ``evaluate``      -- the semantic function IL[[.]] of Fig. 3;
* ``compile_contr`` -- tau_c / tau_e and the smart constructor tplus, Sec. 4;
* ``cut_payoff``    -- cutPayoff, Sec. 4.1.

Readings of passages that are garbled or silent (listed in the design notes):

* loopif (Fig. 3): the recursion reads ``iter(n-1, t0'+1)`` when the
  condition is false and n > 0.  The condition is tested at t0, ..., t0+n
  (n+1 tests); the then-branch is evaluated at the first time it holds, the
  else-branch at t0+n.  The Haskell ``loopif`` and the Futhark while-loop of
  Sec. 6 agree with this reading.
* payoff (Fig. 3): the discount is taken at T[t]delta + t0, i.e. the payoff
  time is shifted by the loopif offset like every other time expression; the
  Futhark output of Sec. 6.2 indexes ``disc[t0]`` inside the loop.
* tau_c(ifWithin(e, t, c1, c2)) (Sec. 4) names c_0, c_1 for the branches;
  read as tau_c(c1), tau_c(c2).
* operator set (open "..." in Sec. 3): unops neg, not; binops add, sub, mult,
  div, lt, le, eq, and, or, max, min.  Values are typed as in Fig. 3:
  nat (from now, texpr, nat literals), real, bool.  Nat subtraction is
  truncated at 0 as in N; div is defined on reals only.
* if (Fig. 3) evaluates only the chosen branch; so does this evaluator, per
  path.  A program whose branches have different types is rejected.

Values are numpy arrays over a set of independent evaluations ("paths"): the
evaluator follows Fig. 3 for each path separately -- every path takes its own
branch of ``if`` and its own iteration count of ``loopif`` -- and merely keeps
paths that are at the same point of the recursion together in one array.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Mapping, Union

import numpy as np

# ---------------------------------------------------------------------------
# Time expressions: TExpr (n | v), ILTExpr (+ tplus), ILTExprZ (+ integers)
# (Sec. 2 Fig. 1 for TExpr; Sec. 3 grammar and Sec. 5 Coq listing for IL).
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class TNum:
    """Integer literal.  Natural in TExpr/ILTExpr, any integer in ILTExprZ."""
    n: int


@dataclass(frozen=True)
class TVar:
    """Template variable, bound by the template environment delta."""
    name: str


@dataclass(frozen=True)
class TPlus:
    """Syntactic addition of two time expressions."""
    a: "TimeExpr"
    b: "TimeExpr"


TimeExpr = Union[TNum, TVar, TPlus]


def tsem(t: TimeExpr, delta: Mapping[str, int]) -> int:
    """T[t]delta (Sec. 2): numerals denote themselves, variables delta(v);
    tplus denotes the sum of its operands."""
    if isinstance(t, TNum):
        return int(t.n)
    if isinstance(t, TVar):
        if t.name not in delta:
            raise KeyError(f"unbound template variable {t.name!r}")
        v = int(delta[t.name])
        if v < 0:
            raise ValueError("template variables range over N")
        return v
    if isinstance(t, TPlus):
        return tsem(t.a, delta) + tsem(t.b, delta)
    raise TypeError(f"not a time expression: {t!r}")


def is_numeral(t: TimeExpr) -> bool:
    return isinstance(t, TNum)


def tplus(t1: TimeExpr, t2: TimeExpr) -> TimeExpr:
    """Smart constructor tplus (Sec. 4): folds two numerals into their sum,
    otherwise builds the syntactic addition."""
    if is_numeral(t1) and is_numeral(t2):
        return TNum(t1.n + t2.n)
    return TPlus(t1, t2)


# ---------------------------------------------------------------------------
# ILExpr (Sec. 3 grammar; Coq definition in Sec. 5)
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Now:
    pass


@dataclass(frozen=True)
class Model:
    label: int
    t: TimeExpr            # ILTExprZ


@dataclass(frozen=True)
class If:
    c: "IL"
    a: "IL"
    b: "IL"


@dataclass(frozen=True)
class LoopIf:
    c: "IL"
    a: "IL"
    b: "IL"
    t: TimeExpr            # TExpr: numeral or variable


@dataclass(frozen=True)
class Payoff:
    t: TimeExpr            # ILTExpr (natural)
    p1: int
    p2: int


@dataclass(frozen=True)
class UnOp:
    op: str
    e: "IL"


@dataclass(frozen=True)
class BinOp:
    op: str
    a: "IL"
    b: "IL"


@dataclass(frozen=True)
class Float:
    f: float


@dataclass(frozen=True)
class Nat:
    n: int


@dataclass(frozen=True)
class Bool:
    b: bool


@dataclass(frozen=True)
class TExp:
    t: TimeExpr            # ILTExpr


IL = Union[Now, Model, If, LoopIf, Payoff, UnOp, BinOp, Float, Nat, Bool, TExp]

UNOPS = ("neg", "not")
BINOPS = ("add", "sub", "mult", "div", "lt", "le", "eq", "and", "or", "max", "min")

# ---------------------------------------------------------------------------
# Semantics IL[[il]]_(rho, delta, t0, t, d, p1, p2)  (Fig. 3)
# ---------------------------------------------------------------------------

REAL = np.float64
BOOL = np.bool_
NAT = np.int64


@dataclass
class Args:
    """The argument vector P-bar = (rho, delta, t0, t, d, p1, p2) of Fig. 3,
    minus t0 which the evaluator threads explicitly.

    ``rho(label, time, idx)`` returns the observable ``label`` at integer
    ``time`` for the evaluations (paths) ``idx`` as a float64 array.
    ``d(time)`` is the discount function N -> R.

    ``margins`` (optional, indexed by path) receives, for every comparison
    of two reals a path evaluates, the smallest |x - y| / max(1, |x|, |y|):
    how far the path's discrete decisions were from a tie.  It does not
    affect the values computed.
    """
    rho: Callable[[int, int, np.ndarray], np.ndarray]
    delta: Mapping[str, int]
    now: int
    d: Callable[[int], float]
    p1: int
    p2: int
    margins: np.ndarray | None = None


def _kind(v: np.ndarray) -> str:
    if v.dtype == REAL:
        return "real"
    if v.dtype == BOOL:
        return "bool"
    if v.dtype == NAT:
        return "nat"
    raise TypeError(f"unexpected value dtype {v.dtype}")


def _unop(op: str, v: np.ndarray) -> np.ndarray:
    k = _kind(v)
    if op == "neg" and k == "real":
        return -v
    if op == "not" and k == "bool":
        return ~v
    raise TypeError(f"{op} undefined on {k}")


def _binop(op: str, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    kx, ky = _kind(x), _kind(y)
    if kx != ky:
        raise TypeError(f"{op} on {kx} and {ky}")
    k = kx
    if k in ("real", "nat"):
        if op == "add":
            return x + y
        if op == "sub":
            return x - y if k == "real" else np.maximum(x - y, 0)
        if op == "mult":
            return x * y
        if op == "div" and k == "real":
            with np.errstate(divide="ignore", invalid="ignore"):
                return x / y
        if op == "lt":
            return x < y
        if op == "le":
            return x <= y
        if op == "eq":
            return x == y
        if op == "max":
            return np.maximum(x, y)
        if op == "min":
            return np.minimum(x, y)
    if k == "bool":
        if op == "and":
            return x & y
        if op == "or":
            return x | y
        if op == "eq":
            return x == y
    raise TypeError(f"{op} undefined on {k}")


def evaluate(il: IL, args: Args, t0: int = 0, idx: np.ndarray | None = None,
             n: int | None = None) -> np.ndarray:
    """IL[[il]] (Fig. 3) for every evaluation in ``idx`` at loop offset t0.

    ``idx`` are the path indices handed to ``rho``; by default ``range(n)``.
    Returns an array of float64 (real), bool or int64 (nat) values.
    """
    if idx is None:
        idx = np.arange(1 if n is None else n)
    return _ev(il, args, int(t0), np.asarray(idx))


def _ev(il: IL, a: Args, t0: int, idx: np.ndarray) -> np.ndarray:
    m = len(idx)
    if isinstance(il, Float):
        return np.full(m, il.f, dtype=REAL)
    if isinstance(il, Bool):
        return np.full(m, bool(il.b), dtype=BOOL)
    if isinstance(il, Nat):
        return np.full(m, int(il.n), dtype=NAT)
    if isinstance(il, TExp):                       # T[t]delta + t0
        return np.full(m, tsem(il.t, a.delta) + t0, dtype=NAT)
    if isinstance(il, Now):                        # t
        return np.full(m, a.now, dtype=NAT)
    if isinstance(il, Model):                      # rho(l, T[t]delta + t0)
        v = np.asarray(a.rho(il.label, tsem(il.t, a.delta) + t0, idx), dtype=REAL)
        if v.shape != (m,):
            raise ValueError("rho returned the wrong shape")
        return v
    if isinstance(il, Payoff):                     # +-d(T[t]delta + t0) or 0
        tp = tsem(il.t, a.delta) + t0
        if (il.p1, il.p2) == (a.p1, a.p2):
            val = a.d(tp)
        elif (il.p1, il.p2) == (a.p2, a.p1):
            val = -a.d(tp)
        else:
            val = 0.0
        return np.full(m, val, dtype=REAL)
    if isinstance(il, UnOp):
        return _unop(il.op, _ev(il.e, a, t0, idx))
    if isinstance(il, BinOp):
        x, y = _ev(il.a, a, t0, idx), _ev(il.b, a, t0, idx)
        if (a.margins is not None and il.op in ("lt", "le", "eq") and x.dtype == REAL
                and y.dtype == REAL and len(idx)):
            gap = np.abs(x - y) / np.maximum(1.0, np.maximum(np.abs(x), np.abs(y)))
            np.minimum.at(a.margins, idx, gap)
        return _binop(il.op, x, y)
    if isinstance(il, If):
        c = _ev(il.c, a, t0, idx)
        if _kind(c) != "bool":
            raise TypeError("if condition must be bool")
        return _merge([(c, il.a, t0), (~c, il.b, t0)], a, idx)
    if isinstance(il, LoopIf):
        return _loopif(il, a, t0, idx)
    raise TypeError(f"not an IL expression: {il!r}")


def _merge(parts, a: Args, idx: np.ndarray) -> np.ndarray:
    """Evaluate each branch only on the paths that chose it and put the
    results back in path order."""
    out = None
    for mask, expr, t0 in parts:
        sel = np.nonzero(mask)[0]
        if len(sel) == 0:
            continue
        v = _ev(expr, a, t0, idx[sel])
        if out is None:
            out = np.empty(len(idx), dtype=v.dtype)
        elif out.dtype != v.dtype:
            raise TypeError("branches of different types")
        out[sel] = v
    if out is None:          # no paths at all
        out = np.empty(0, dtype=REAL)
    return out


def _loopif(il: LoopIf, a: Args, t0: int, idx: np.ndarray) -> np.ndarray:
    """iter(T[t]delta, t0) of Fig. 3, with the reading given in the module
    docstring: test at t0+k for k = 0..n, then-branch at the first k whose
    test holds, else-branch at t0+n."""
    n = tsem(il.t, a.delta)
    out = None
    pending = np.arange(len(idx))                  # positions still iterating

    def put(pos, v):
        nonlocal out
        if out is None:
            out = np.empty(len(idx), dtype=v.dtype)
        elif out.dtype != v.dtype:
            raise TypeError("loopif branches of different types")
        out[pos] = v

    for k in range(n + 1):
        if len(pending) == 0:
            break
        c = _ev(il.c, a, t0 + k, idx[pending])
        if _kind(c) != "bool":
            raise TypeError("loopif condition must be bool")
        hit = pending[c]
        if len(hit):
            put(hit, _ev(il.a, a, t0 + k, idx[hit]))
        pending = pending[~c]
    if len(pending):
        put(pending, _ev(il.b, a, t0 + n, idx[pending]))
    if out is None:
        out = np.empty(0, dtype=REAL)
    return out


# ---------------------------------------------------------------------------
# cutPayoff (Sec. 4.1)
# ---------------------------------------------------------------------------


def cut_payoff(il: IL) -> IL:
    """cutPayoff (Sec. 4.1): every payoff(t, p1, p2) becomes
    if(t < now, 0, payoff(t, p1, p2)); all other constructs are rebuilt from
    their transformed sub-expressions (loopif included, whose case the
    printed definition leaves implicit); leaves are unchanged."""
    if isinstance(il, Payoff):
        return If(BinOp("lt", TExp(il.t), Now()), Float(0.0), il)
    if isinstance(il, UnOp):
        return UnOp(il.op, cut_payoff(il.e))
    if isinstance(il, BinOp):
        return BinOp(il.op, cut_payoff(il.a), cut_payoff(il.b))
    if isinstance(il, If):
        return If(cut_payoff(il.c), cut_payoff(il.a), cut_payoff(il.b))
    if isinstance(il, LoopIf):
        return LoopIf(cut_payoff(il.c), cut_payoff(il.a), cut_payoff(il.b), il.t)
    return il


def loopif0_to_if(il: IL) -> IL:
    """The Sec. 6.1 rewrite of loopif with a literal 0 bound into if."""
    if isinstance(il, LoopIf):
        c, a_, b = loopif0_to_if(il.c), loopif0_to_if(il.a), loopif0_to_if(il.b)
        if isinstance(il.t, TNum) and il.t.n == 0:
            return If(c, a_, b)
        return LoopIf(c, a_, b, il.t)
    if isinstance(il, If):
        return If(loopif0_to_if(il.c), loopif0_to_if(il.a), loopif0_to_if(il.b))
    if isinstance(il, UnOp):
        return UnOp(il.op, loopif0_to_if(il.e))
    if isinstance(il, BinOp):
        return BinOp(il.op, loopif0_to_if(il.a), loopif0_to_if(il.b))
    return il


def size(il: IL) -> int:
    """Number of IL nodes (time expressions not counted)."""
    if isinstance(il, (If, LoopIf)):
        return 1 + size(il.c) + size(il.a) + size(il.b)
    if isinstance(il, UnOp):
        return 1 + size(il.e)
    if isinstance(il, BinOp):
        return 1 + size(il.a) + size(il.b)
    return 1
