"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every entry point of include/pc.h, the text assembler matches an
encoder written from the header's bytecode description, and the verifier
rejects malformed programs with the documented status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import il, il_text
import workloads as W

pc = pytest.importorskip("paper_2108_03076_gb300")


@pytest.fixture(scope="session", autouse=True)
def built():
    from paper_2108_03076_gb300 import build
    build.build()
    return pc.lib()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "pc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:pc_status|const char \*)\s*(pc_\w+)\s*\(", txt, re.M)))


def test_exports_every_declared_symbol():
    names = header_symbols()
    assert len(names) >= 16
    L = ctypes.CDLL(pc.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(pc.EXPORTED)


# --- an encoder of the documented bytecode format (test-side) --------------

OPS = {"now": 4, "texpr": 5, "model": 6, "payoff": 7, "neg": 8, "not": 9, "add": 10,
       "sub": 11, "mult": 12, "div": 13, "lt": 14, "le": 15, "eq": 16, "and": 17, "or": 18,
       "max": 19, "min": 20, "if": 21, "loopif": 22}


def _terms(t):
    if isinstance(t, il.TNum):
        return [t.n & 0x7FFFFFFF]
    if isinstance(t, il.TVar):
        return [0x80000000 | int(t.name[1:])]
    return _terms(t.a) + _terms(t.b)


def encode(e, consts):
    def T(t):
        ts = _terms(t)
        return [len(ts)] + ts
    if isinstance(e, il.Float):
        if e.f not in consts:
            consts.append(e.f)
        return [1 | (consts.index(e.f) << 8)]
    if isinstance(e, il.Bool):
        return [2 | (int(e.b) << 8)]
    if isinstance(e, il.Nat):
        return [3 | (e.n << 8)]
    if isinstance(e, il.Now):
        return [4]
    if isinstance(e, il.TExp):
        return [5] + T(e.t)
    if isinstance(e, il.Model):
        return [6 | (e.label << 8)] + T(e.t)
    if isinstance(e, il.Payoff):
        return [7, e.p1 & 0xFFFFFFFF, e.p2 & 0xFFFFFFFF] + T(e.t)
    if isinstance(e, il.UnOp):
        return encode(e.e, consts) + [OPS[e.op]]
    if isinstance(e, il.BinOp):
        return encode(e.a, consts) + encode(e.b, consts) + [OPS[e.op]]
    if isinstance(e, il.If):
        return encode(e.c, consts) + encode(e.a, consts) + encode(e.b, consts) + [21]
    if isinstance(e, il.LoopIf):
        return encode(e.c, consts) + encode(e.a, consts) + encode(e.b, consts) + [22] + T(e.t)
    raise TypeError(e)


TEXTS = [
    W.european_text(100.0), W.european_if_text(100.0), W.digital_text(95.5),
    W.zero_coupon_text(), W.exchange_text(), W.autocall_text([1.0, 1.0, 1.0]),
    W.barrier_ladder_text([1.0, 2.0, 3.0]),
    "(add (if (lt (texpr (tplus $1 -0)) (now)) 0.0 (payoff (tplus $0 3) 0 1)) (mult (model 2 -4) 1e-3))",
    "(loopif (and #t (not #f)) (neg (model 0 (tplus 2 (tplus $0 $1)))) (max 1.5 -2.25) $3)",
    "(if (eq (nat 5) (texpr 5)) 1.0 (min 2.0 3.0)) ; comment\n",
]


@pytest.mark.parametrize("text", TEXTS)
def test_assembler_matches_documented_encoding(text):
    words, consts = pc.pc_assemble(text)
    want_consts = []
    want = encode(il_text.parse(text), want_consts)
    assert list(words) == want
    assert list(consts) == want_consts


@pytest.mark.parametrize("text,msg", [("(add 1.0)", "bad literal"), ("(foo 1.0 2.0)", "unknown"),
                                      ("1", "bad literal"), ("(model 9 0)", "label"),
                                      ("(add 1.0 2.0) 3.0", "trailing")])
def test_assembler_syntax_errors(text, msg):
    with pytest.raises(pc.PcError) as ei:
        pc.pc_assemble(text)
    assert ei.value.name == "PC_ESYNTAX" and msg in str(ei.value)


def verify(text, tparams=()):
    w, k = pc.pc_assemble(text)
    return pc.pc_verify_payoff(w, k, tparams)


def test_verifier_accepts_workloads_and_reports_structure():
    info = verify(W.barrier_ladder_text([1.0, 1.0, 1.0]), [365])
    assert info.n_nodes == il.size(il_text.parse(W.barrier_ladder_text([1.0] * 3)))
    assert info.n_loops == 1 and info.result_is_real == 1 and info.n_tparams_used == 1
    info = verify(W.autocall_text([1.0] * 3))
    assert info.n_loops == 0              # loopif(.., 0) runs as if


@pytest.mark.parametrize("text,tp,status", [
    ("(lt 1.0 2.0)", (), "PC_EBYTECODE"),                   # result must be real
    ("(add 1.0 (nat 1))", (), "PC_EBYTECODE"),             # mixed types
    ("(if 1.0 2.0 3.0)", (), "PC_EBYTECODE"),              # non-bool condition
    ("(if #t 2.0 #f)", (), "PC_EBYTECODE"),                # branches differ
    ("(div (nat 4) (nat 2))", (), "PC_EBYTECODE"),
    ("(payoff $2 0 1)", (1, 2), "PC_ETPARAM"),             # unbound
    ("(payoff $0 0 1)", (-1,), "PC_ETPARAM"),              # negative
    ("(payoff -1 0 1)", (), "PC_EBYTECODE"),               # natural time
])
def test_verifier_rejects(text, tp, status):
    with pytest.raises(pc.PcError) as ei:
        verify(text, tp)
    assert ei.value.name == status


def test_verifier_rejects_malformed_words():
    w, k = pc.pc_assemble("(add 1.0 2.0)")
    for bad, status in [(w[:-1], "PC_EBYTECODE"),                       # leftover values
                        (np.append(w, 10), "PC_EBYTECODE"),             # underflow
                        (np.array([99], np.uint32), "PC_EBYTECODE"),    # bad opcode
                        (np.array([1 | (5 << 8)], np.uint32), "PC_EBYTECODE")]:  # const index
        with pytest.raises(pc.PcError) as ei:
            pc.pc_verify_payoff(bad, k, ())
        assert ei.value.name == status
    with pytest.raises(pc.PcError) as ei:
        pc.pc_verify_payoff(np.array([6, 1], np.uint32), k, ())     # truncated time
    assert ei.value.name == "PC_EBYTECODE"
