"""pc_cut_payoff (cutPayoff, Sec. 4.1, in the library) against the oracle's
cut_payoff: on every parity case the library's transformed bytecode and the
oracle's transformed IL (printed, then assembled) load to the same
executable program, and a program without payoffs is unchanged."""
import numpy as np
import pytest

from cases import CASES
import paper_2108_03076_gb300 as pc
from oracle import il, il_text

PARAMS = [f"${i}" for i in range(8)]


@pytest.mark.parametrize("name", sorted(CASES))
def test_cut_payoff_matches_oracle(name):
    text, tp, _, _ = CASES[name]
    w, k = pc.pc_assemble(text)
    cw, ck = pc.pc_cut_payoff(w, k)
    rw, rk = pc.pc_assemble(il_text.to_text(il.cut_payoff(il_text.parse(text)), PARAMS))
    got, want = pc.pc_debug_program(cw, ck, tp), pc.pc_debug_program(rw, rk, tp)
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)
    # one if(t < now, 0, .) per payoff: six more words per payoff word group
    n_payoff = text.count("(payoff")
    assert len(cw) > len(w) or n_payoff == 0


def test_cut_payoff_without_payoffs_is_identity():
    w, k = pc.pc_assemble("(add (model 0 1) 2.5)")
    cw, ck = pc.pc_cut_payoff(w, k)
    np.testing.assert_array_equal(cw, w)
    np.testing.assert_array_equal(ck, k)


def test_cut_payoff_reuses_a_zero_literal_and_rejects_bad_bytecode():
    w, k = pc.pc_assemble("(add 0.0 (mult (model 0 1) (payoff 1 0 1)))")
    cw, ck = pc.pc_cut_payoff(w, k)
    np.testing.assert_array_equal(ck, k)          # 0.0 was there already
    with pytest.raises(pc.PcError) as ei:
        pc.pc_cut_payoff(np.array([99], np.uint32), np.zeros(0))
    assert ei.value.name == "PC_EBYTECODE"
