"""Textual S-expression form of IL: printer and parser (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The text form is an interface format shared with the product's assembler;
each side has its own printer/parser.  Grammar (one construct per IL node of
Sec. 3):

    il  ::= (now) | (model L tz) | (if il il il) | (loopif il il il t)
          | (payoff t P P) | (texpr t) | (neg il) | (not il)
          | (BINOP il il) | REAL | #t | #f | (nat N)
    t   ::= INT | $K | (tplus t t)       ; $K = template variable number K
    BINOP ::= add sub mult div lt le eq and or max min

REAL literals always contain '.', 'e' or 'E' (Python ``repr`` of a float,
which round-trips exactly); labels and parties are integers; ``;`` starts a
comment.  Template variable names map to ``$K`` through an ordered list.
"""
from __future__ import annotations

from typing import List, Sequence

from .il import (IL, BINOPS, UNOPS, Bool, BinOp, Float, If, LoopIf, Model, Nat,
                 Now, Payoff, TExp, TimeExpr, TNum, TPlus, TVar, UnOp)


def time_to_text(t: TimeExpr, params: Sequence[str]) -> str:
    if isinstance(t, TNum):
        return str(int(t.n))
    if isinstance(t, TVar):
        return f"${list(params).index(t.name)}"
    if isinstance(t, TPlus):
        return f"(tplus {time_to_text(t.a, params)} {time_to_text(t.b, params)})"
    raise TypeError(t)


def to_text(il: IL, params: Sequence[str] = ()) -> str:
    """Print an IL tree; template variable ``params[k]`` prints as ``$k``."""
    T = lambda t: time_to_text(t, params)
    if isinstance(il, Float):
        r = repr(float(il.f))
        if not any(ch in r for ch in ".eE"):
            r += ".0"
        return r
    if isinstance(il, Bool):
        return "#t" if il.b else "#f"
    if isinstance(il, Nat):
        return f"(nat {int(il.n)})"
    if isinstance(il, Now):
        return "(now)"
    if isinstance(il, TExp):
        return f"(texpr {T(il.t)})"
    if isinstance(il, Model):
        return f"(model {il.label} {T(il.t)})"
    if isinstance(il, Payoff):
        return f"(payoff {T(il.t)} {il.p1} {il.p2})"
    if isinstance(il, UnOp):
        return f"({il.op} {to_text(il.e, params)})"
    if isinstance(il, BinOp):
        return f"({il.op} {to_text(il.a, params)} {to_text(il.b, params)})"
    if isinstance(il, If):
        return f"(if {to_text(il.c, params)} {to_text(il.a, params)} {to_text(il.b, params)})"
    if isinstance(il, LoopIf):
        return (f"(loopif {to_text(il.c, params)} {to_text(il.a, params)} "
                f"{to_text(il.b, params)} {T(il.t)})")
    raise TypeError(il)


def _tokens(s: str) -> List[str]:
    out: List[str] = []
    for line in s.splitlines():
        line = line.split(";", 1)[0]
        out.extend(line.replace("(", " ( ").replace(")", " ) ").split())
    return out


class _Parser:
    def __init__(self, text: str, params: Sequence[str] | None):
        self.toks = _tokens(text)
        self.i = 0
        self.params = params

    def peek(self) -> str:
        if self.i >= len(self.toks):
            raise ValueError("unexpected end of IL text")
        return self.toks[self.i]

    def next(self) -> str:
        t = self.peek()
        self.i += 1
        return t

    def expect(self, tok: str) -> None:
        t = self.next()
        if t != tok:
            raise ValueError(f"expected {tok!r}, got {t!r}")

    def int_(self) -> int:
        return int(self.next())

    def time(self) -> TimeExpr:
        t = self.next()
        if t == "(":
            self.expect("tplus")
            a = self.time()
            b = self.time()
            self.expect(")")
            return TPlus(a, b)
        if t.startswith("$"):
            k = int(t[1:])
            name = self.params[k] if self.params is not None else f"${k}"
            return TVar(name)
        return TNum(int(t))

    def il(self) -> IL:
        t = self.next()
        if t == "#t":
            return Bool(True)
        if t == "#f":
            return Bool(False)
        if t != "(":
            if not any(ch in t for ch in ".eE") or t.startswith("$"):
                raise ValueError(f"bad literal {t!r}")
            return Float(float(t))
        head = self.next()
        if head == "now":
            out: IL = Now()
        elif head == "nat":
            out = Nat(self.int_())
        elif head == "texpr":
            out = TExp(self.time())
        elif head == "model":
            lab = self.int_()
            out = Model(lab, self.time())
        elif head == "payoff":
            tt = self.time()
            out = Payoff(tt, self.int_(), self.int_())
        elif head in UNOPS:
            out = UnOp(head, self.il())
        elif head in BINOPS:
            a = self.il()
            out = BinOp(head, a, self.il())
        elif head == "if":
            c = self.il()
            a = self.il()
            out = If(c, a, self.il())
        elif head == "loopif":
            c = self.il()
            a = self.il()
            b = self.il()
            out = LoopIf(c, a, b, self.time())
        else:
            raise ValueError(f"unknown construct {head!r}")
        self.expect(")")
        return out


def parse(text: str, params: Sequence[str] | None = None) -> IL:
    """Parse one IL expression; ``$k`` becomes TVar(params[k]) (or "$k")."""
    p = _Parser(text, params)
    out = p.il()
    if p.i != len(p.toks):
        raise ValueError("trailing tokens after IL expression")
    return out
