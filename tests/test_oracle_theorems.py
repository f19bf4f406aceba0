"""The paper's theorems as executable pins of the oracle, checked by brute
force over random small contracts and enumerated environments:

* Theorem 1 (i)/(ii), Sec. 4: compiled expressions evaluate to the CL value;
  the compiled contract evaluates to the discounted sum of its trace;
* Theorem 5, Sec. 4.1: cutPayoff evaluated at now = n equals the discounted
  trace summed from n;
* instantiation soundness (Lemma 2, Sec. 2) and TC(inst(c, delta));
* invariants: zero pays 0, scale and both are linear, translate delays.
"""
import itertools
import random

import numpy as np
import pytest

from oracle import cl, il
from oracle.cl import (BLit, Both, IfWithin, Obs, Op, RLit, Scale, Transfer, Translate,
                       Zero, csem, esem, horizon, inst, trace_flow)
from oracle.il import TNum, TVar

VALS = (80.0, 100.0, 120.0)
LABELS = (0, 1)
DELTA = {"u": 1, "w": 2}


def rand_time(rng):
    return rng.choice([TNum(0), TNum(1), TNum(2), TVar("u"), TVar("w")])


def rand_real(rng, depth):
    if depth <= 0 or rng.random() < 0.3:
        if rng.random() < 0.5:
            return Obs(rng.choice(LABELS), rng.choice([-1, 0, 0, 1]))
        return RLit(rng.choice([0.5, 1.0, 2.0, 100.0]))
    k = rng.random()
    if k < 0.55:
        return Op(rng.choice(["add", "sub", "mult", "max", "min"]),
                  (rand_real(rng, depth - 1), rand_real(rng, depth - 1)))
    if k < 0.7:
        return Op("div", (rand_real(rng, depth - 1), RLit(rng.choice([2.0, 4.0, 100.0]))))
    if k < 0.8:
        return Op("neg", (rand_real(rng, depth - 1),))
    return Op("cond", (rand_bool(rng, depth - 1), rand_real(rng, depth - 1),
                       rand_real(rng, depth - 1)))


def rand_bool(rng, depth):
    if depth <= 0 or rng.random() < 0.2:
        if rng.random() < 0.2:
            return BLit(rng.random() < 0.5)
        return Op(rng.choice(["lt", "le"]), (Obs(rng.choice(LABELS), rng.choice([-1, 0, 1])),
                                            RLit(rng.choice(VALS))))
    k = rng.random()
    if k < 0.4:
        return Op(rng.choice(["lt", "le", "eq"]), (rand_real(rng, depth - 1),
                                                  rand_real(rng, depth - 1)))
    if k < 0.8:
        return Op(rng.choice(["and", "or"]), (rand_bool(rng, depth - 1), rand_bool(rng, depth - 1)))
    return Op("not", (rand_bool(rng, depth - 1),))


def rand_contr(rng, depth):
    if depth <= 0 or rng.random() < 0.15:
        return rng.choice([Zero(), Transfer(0, 1), Transfer(1, 0), Transfer(0, 2)])
    k = rng.random()
    if k < 0.25:
        return Scale(rand_real(rng, 2), rand_contr(rng, depth - 1))
    if k < 0.45:
        return Translate(rand_time(rng), rand_contr(rng, depth - 1))
    if k < 0.65:
        return Both(rand_contr(rng, depth - 1), rand_contr(rng, depth - 1))
    return IfWithin(rand_bool(rng, 2), rand_time(rng), rand_contr(rng, depth - 1),
                    rand_contr(rng, depth - 1))


def env_table(rng, n_env, t_lo, t_hi):
    """Random environments: values[env, label, time - t_lo]."""
    return np.array([[[rng.choice(VALS) for _ in range(t_lo, t_hi + 1)] for _ in LABELS]
                     for _ in range(n_env)])


def disc(t):
    return 0.95 ** t * (1.0 + 0.01 * t)


def il_args(table, t_lo, delta, now=0, p1=0, p2=1):
    return il.Args(rho=lambda l, t, idx: table[idx, l, t - t_lo], delta=delta, now=now,
                   d=disc, p1=p1, p2=p2)


def cl_env(table, e, t_lo):
    return lambda l, t: float(table[e, l, t - t_lo])


CONTRACTS = [rand_contr(random.Random(1000 + s), 4) for s in range(60)]


@pytest.mark.parametrize("k", range(len(CONTRACTS)))
def test_theorem1_ii_and_theorem5(k):
    c = CONTRACTS[k]
    rng = random.Random(7 + k)
    H = horizon(c, DELTA)
    t_lo, t_hi = -2, H + 3
    table = env_table(rng, 40, t_lo, t_hi)
    compiled = cl.compile_contr(c)
    cut = il.cut_payoff(compiled)
    for p1, p2 in [(0, 1), (1, 0), (0, 2)]:
        got = il.evaluate(compiled, il_args(table, t_lo, DELTA, 0, p1, p2), idx=np.arange(len(table)))
        for e in range(len(table)):
            tr = csem(c, cl_env(table, e, t_lo), DELTA)
            want = sum(disc(t) * trace_flow(tr, t, p1, p2) for t in range(H + 1))
            assert got[e] == pytest.approx(want, rel=1e-12, abs=1e-12)
            assert all(t <= H for t in tr)
        # Theorem 5: cutPayoff at now = n sums the trace from n
        for n in range(H + 2):
            gotc = il.evaluate(cut, il_args(table, t_lo, DELTA, n, p1, p2), idx=np.arange(len(table)))
            for e in range(0, len(table), 7):
                tr = csem(c, cl_env(table, e, t_lo), DELTA)
                want = sum(disc(t) * trace_flow(tr, t, p1, p2) for t in range(n, H + 1))
                assert gotc[e] == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_theorem1_i_expressions():
    rng = random.Random(99)
    table = env_table(rng, 30, -2, 2)
    for s in range(150):
        e = rand_real(rng, 4) if s % 2 else rand_bool(rng, 4)
        got = il.evaluate(cl.compile_exp(e, TNum(0)), il_args(table, -2, DELTA),
                          idx=np.arange(len(table)))
        for k in range(len(table)):
            want = esem(e, cl_env(table, k, -2))
            if isinstance(want, bool):
                assert bool(got[k]) == want
            elif np.isfinite(want):
                assert got[k] == pytest.approx(want, rel=1e-13, abs=1e-13)


def test_theorem1_ii_enumerated_environments():
    """All environments over one label, times -1..4, values {80, 100, 120}."""
    c = IfWithin(Op("lt", (Obs(0, 0), RLit(100.0))), TVar("w"),
                 Scale(Obs(0, -1), Transfer(0, 1)),
                 Translate(TNum(1), Scale(Op("sub", (Obs(0, 0), Obs(0, -1))), Transfer(1, 0))))
    t_lo, t_hi = -1, 4
    combos = np.array(list(itertools.product(VALS, repeat=t_hi - t_lo + 1)))
    table = np.stack([combos, combos], axis=1)
    H = horizon(c, DELTA)
    got = il.evaluate(cl.compile_contr(c), il_args(table, t_lo, DELTA), idx=np.arange(len(table)))
    for e in range(len(table)):
        tr = csem(c, cl_env(table, e, t_lo), DELTA)
        want = sum(disc(t) * trace_flow(tr, t, 0, 1) for t in range(H + 1))
        assert got[e] == pytest.approx(want, rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("k", range(0, len(CONTRACTS), 3))
def test_instantiation_soundness(k):
    c = CONTRACTS[k]
    ci = inst(c, DELTA)
    assert cl.template_closed(ci)
    rng = random.Random(k)
    H = horizon(c, DELTA)
    table = env_table(rng, 10, -2, H + 3)
    for e in range(len(table)):
        rho = cl_env(table, e, -2)
        assert csem(c, rho, DELTA) == csem(ci, rho, {"u": 77, "w": 99})


def _value(c, table, t_lo=-2, delta=DELTA, d=disc):
    a = il.Args(rho=lambda l, t, idx: table[idx, l, t - t_lo], delta=delta, now=0, d=d,
                p1=0, p2=1)
    return il.evaluate(cl.compile_contr(c), a, idx=np.arange(len(table)))


def test_invariants_zero_scale_both_translate():
    rng = random.Random(5)
    for k in range(0, len(CONTRACTS), 2):
        c, c2 = CONTRACTS[k], CONTRACTS[k + 1]
        H = max(horizon(c, DELTA), horizon(c2, DELTA))
        table = env_table(rng, 25, -2, H + 6)
        v, v2 = _value(c, table), _value(c2, table)
        np.testing.assert_allclose(_value(Scale(RLit(2.5), c), table), 2.5 * v, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(_value(Both(c, c2), table), v + v2, rtol=1e-13, atol=1e-13)
        # translate(3, c) in env rho with discount d == c in rho/3 with d/3
        shifted = table[:, :, 3:]
        v_shift = _value(c, shifted, d=lambda t: disc(t + 3))
        np.testing.assert_allclose(_value(Translate(TNum(3), c), table), v_shift,
                                   rtol=1e-13, atol=1e-13)
    assert (_value(Zero(), env_table(rng, 3, -2, 2)) == 0.0).all()
