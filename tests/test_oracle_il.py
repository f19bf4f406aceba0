"""Pins of the oracle's IL semantics, compiler and cutPayoff against the
paper's worked examples (Sec. 4 Examples 3-4, Sec. 6.2 barrier listing)."""
import itertools

import numpy as np
import pytest

from conftest import read_golden
from oracle import cl, il, il_text
from oracle.cl import IfWithin, Obs, RLit, Scale, Transfer, Translate, Zero, Both, gt, op
from oracle.il import TNum, TPlus, TVar

YOU, ME, AAPL = 0, 1, 0


def example3_contract():
    """Sec. 4, Example 3."""
    t0, t1 = TVar("t0"), TVar("t1")
    return Translate(t0, Both(
        Scale(RLit(100.0), Transfer(YOU, ME)),
        Translate(t1, IfWithin(gt(Obs(AAPL, 0), RLit(100.0)), TNum(0),
                               Scale(op("sub", Obs(AAPL, 0), RLit(100.0)), Transfer(YOU, ME)),
                               Zero()))))


def norm_time(t):
    """Canonical form of a time expression: (integer sum, sorted variables)."""
    if isinstance(t, TNum):
        return (t.n, ())
    if isinstance(t, TVar):
        return (0, (t.name,))
    a, b = norm_time(t.a), norm_time(t.b)
    return (a[0] + b[0], tuple(sorted(a[1] + b[1])))


def norm(e):
    """Replace every time expression by its canonical form."""
    if isinstance(e, il.Model):
        return ("model", e.label, norm_time(e.t))
    if isinstance(e, il.Payoff):
        return ("payoff", norm_time(e.t), e.p1, e.p2)
    if isinstance(e, il.TExp):
        return ("texpr", norm_time(e.t))
    if isinstance(e, il.LoopIf):
        return ("loopif", norm(e.c), norm(e.a), norm(e.b), norm_time(e.t))
    if isinstance(e, il.If):
        return ("if", norm(e.c), norm(e.a), norm(e.b))
    if isinstance(e, il.BinOp):
        return (e.op, norm(e.a), norm(e.b))
    if isinstance(e, il.UnOp):
        return (e.op, norm(e.e))
    return e


PARAMS = ["t0", "t1"]


def test_compile_example3_structure():
    got = cl.compile_contr(example3_contract())
    want = il_text.parse(read_golden("compile_example.il"), PARAMS)
    assert got == want


def test_compile_example3_matches_printed_form():
    got = il.loopif0_to_if(cl.compile_contr(example3_contract()))
    printed = il_text.parse(read_golden("compile_example_printed.il"), PARAMS)
    assert norm(got) == norm(printed)


def test_cutpayoff_example4():
    e = cl.compile_contr(example3_contract())
    got = il.loopif0_to_if(il.cut_payoff(e))
    want = il_text.parse(read_golden("cutpayoff_example.il"), PARAMS)
    assert norm(got) == norm(want)


def test_smart_tplus_folds_numerals_only():
    assert il.tplus(TNum(2), TNum(3)) == TNum(5)
    assert il.tplus(TNum(0), TVar("v")) == TPlus(TNum(0), TVar("v"))
    assert il.tplus(TNum(4), TNum(-1)) == TNum(3)
    # a translate chain of numerals folds to one numeral (Sec. 4, Remark 1)
    c = Translate(TNum(2), Translate(TNum(3), Transfer(0, 1)))
    assert cl.compile_contr(c) == il.Payoff(TNum(5), 0, 1)


def _futhark_barrier(ext, disc, T):
    """The while-loop of the Futhark listing in Sec. 6.2: advance t0 while the
    barrier test fails and t0 is below the window end (the bound read as
    start + window), then pay 0 if the test holds at t0, else 2000 * disc[t0]."""
    t0 = 0
    while (not (ext[t0] <= 4000.0)) and t0 < 0 + T:
        t0 += 1
    return 0.0 if ext[t0] <= 4000.0 else 2000.0 * disc[t0]


@pytest.mark.parametrize("T", [0, 1, 2, 3])
def test_loopif_matches_futhark_while_loop(T):
    prog = il_text.parse(read_golden("barrier_loopif.il"), ["t"])
    vals = [3900.0, 4000.0, 4100.0]
    horizon = T + 1
    envs = np.array(list(itertools.product(vals, repeat=horizon)))   # [env, time]
    disc = [0.9 ** k + 0.01 * k for k in range(horizon)]
    args = il.Args(rho=lambda l, t, idx: envs[idx, t], delta={"t": T}, now=0,
                   d=lambda t: disc[t], p1=0, p2=1)
    got = il.evaluate(prog, args, idx=np.arange(len(envs)))
    want = [_futhark_barrier(e, disc, T) for e in envs]
    np.testing.assert_array_equal(got, want)


def test_loopif_tests_window_inclusive_and_else_at_end():
    # cond true only at time 3: with window 3 the then-branch runs at t0 = 3;
    # with window 2 the else-branch runs at t0 = 2.
    prog = il.LoopIf(il.BinOp("eq", il.TExp(TNum(0)), il.Nat(3)),
                     il.TExp(TNum(0)), il.BinOp("add", il.TExp(TNum(0)), il.Nat(100)),
                     TVar("n"))
    a = lambda n: il.Args(rho=None, delta={"n": n}, now=0, d=None, p1=0, p2=1)
    assert il.evaluate(prog, a(3))[0] == 3
    assert il.evaluate(prog, a(2))[0] == 102
    assert il.evaluate(prog, a(0))[0] == 100


def test_payoff_inside_loopif_is_shifted():
    # payoff(0) inside the then-branch of a loopif firing at offset 2 is
    # discounted at time 2 (Sec. 6.2 listing indexes disc[t0]).
    prog = il.LoopIf(il.BinOp("le", il.Nat(2), il.TExp(TNum(0))),
                     il.Payoff(TNum(0), 0, 1), il.Float(-1.0), TNum(5))
    args = il.Args(rho=None, delta={}, now=0, d=lambda t: 10.0 ** -t, p1=0, p2=1)
    assert il.evaluate(prog, args)[0] == pytest.approx(1e-2)


def test_payoff_parties_sign():
    d = lambda t: 0.5
    for (q1, q2, want) in [(0, 1, 0.5), (1, 0, -0.5), (0, 2, 0.0), (2, 2, 0.0)]:
        args = il.Args(rho=None, delta={}, now=0, d=d, p1=0, p2=1)
        assert il.evaluate(il.Payoff(TNum(0), q1, q2), args)[0] == want


def test_now_texpr_and_nat_ops():
    args = il.Args(rho=None, delta={"v": 4}, now=7, d=None, p1=0, p2=1)
    e = il.BinOp("sub", il.TExp(TPlus(TVar("v"), TNum(1))), il.Now())   # 5 - 7 truncated
    assert il.evaluate(e, args)[0] == 0
    e = il.BinOp("lt", il.TExp(TVar("v")), il.Now())
    assert bool(il.evaluate(e, args)[0]) is True
    assert il.evaluate(il.TExp(TVar("v")), args, t0=3)[0] == 7


def test_if_evaluates_only_the_chosen_branch():
    # the untaken branch is ill-typed; Fig. 3 never evaluates it
    bad = il.BinOp("add", il.Float(1.0), il.Bool(True))
    args = il.Args(rho=None, delta={}, now=0, d=None, p1=0, p2=1)
    assert il.evaluate(il.If(il.Bool(True), il.Float(2.0), bad), args)[0] == 2.0
    with pytest.raises(TypeError):
        il.evaluate(il.If(il.Bool(False), il.Float(2.0), bad), args)


def test_type_errors():
    args = il.Args(rho=None, delta={}, now=0, d=None, p1=0, p2=1)
    for e in [il.BinOp("add", il.Float(1.0), il.Nat(1)), il.UnOp("not", il.Float(1.0)),
              il.If(il.Float(1.0), il.Float(1.0), il.Float(2.0)),
              il.BinOp("div", il.Nat(4), il.Nat(2))]:
        with pytest.raises(TypeError):
            il.evaluate(e, args)


def test_text_round_trip_of_workload_programs():
    import workloads as W
    texts = [W.european_text(100.0), W.autocall_text([1.0, 1.0, 1.0]),
             W.barrier_ladder_text([1.0, 1.0, 1.0]), W.exchange_text()]
    for t in texts:
        e = il_text.parse(t, ["T"])
        assert il_text.parse(il_text.to_text(e, ["T"]), ["T"]) == e
