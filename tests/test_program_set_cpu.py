"""Host-side packing of pc_load_payoffs' arguments (ProgramSet): the
programs' words, literals and template parameters concatenated, with
offset arrays of n + 1 entries that recover each program."""
import numpy as np

import paper_2108_03076_gb300 as pc
import workloads as W


def test_program_set_offsets_recover_every_program():
    progs = []
    for it in W.portfolio()[:25]:
        w, k = pc.pc_assemble(it.il_text)
        progs.append((w, k, it.tparams))
    progs.append((progs[0][0], np.zeros(0), []))          # no literals, no parameters
    ps = pc.ProgramSet(progs)
    assert ps.n == len(progs)
    for off in (ps.word_off, ps.const_off, ps.param_off):
        assert off.dtype == np.uintp and off.size == ps.n + 1 and off[0] == 0
        assert np.all(np.diff(off.astype(np.int64)) >= 0)
    for i, (w, k, t) in enumerate(progs):
        np.testing.assert_array_equal(ps.words[ps.word_off[i]:ps.word_off[i + 1]], np.asarray(w, np.uint32))
        np.testing.assert_array_equal(ps.consts[ps.const_off[i]:ps.const_off[i + 1]], np.asarray(k, np.float64))
        np.testing.assert_array_equal(ps.params[ps.param_off[i]:ps.param_off[i + 1]], np.asarray(t, np.int32))
    assert ps.words.dtype == np.uint32 and ps.consts.dtype == np.float64 and ps.params.dtype == np.int32


def test_load_payoffs_refuses_a_null_context():
    w, k = pc.pc_assemble(W.portfolio()[0].il_text)
    try:
        pc.pc_load_payoffs(0, [(w, k, [])])
    except pc.PcError as e:
        assert e.name == "PC_EINVAL"
    else:
        raise AssertionError("a null context must be refused")
