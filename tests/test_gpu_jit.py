"""GPU run-time specialised kernels (pc_set_jit): the same per-path payoffs,
bit for bit, and the same sums as the interpreting kernel on every test
program, the oracle's values on a sample, the compiled kernel reused when
the same program is loaded again, the same again for launches whose
window of dates lives in HBM, and programs beyond the specialising limit
interpreted."""
import time

import numpy as np
import pytest

from cases import CASES
from gpu_common import Engine, compare, oracle_paths, torch
import paper_2108_03076_gb300 as pc
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    yield e
    pc.pc_set_jit(e.ctx, False)
    e.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_specialised_equals_interpreter(eng, name):
    text, tp, spec, notional = CASES[name]
    m, k = eng.model(spec), eng.contract(text, tp)
    n, seed = 4096 + 37, 0xABC + len(name)
    pc.pc_set_jit(eng.ctx, False)
    x0, s0 = eng.paths(m, k, n, seed)
    pc.pc_set_jit(eng.ctx, True)
    try:
        x1, s1 = eng.paths(m, k, n, seed)
        a1 = eng.sums(m, k, 1 << 16, seed)
    finally:
        pc.pc_set_jit(eng.ctx, False)
    a0 = eng.sums(m, k, 1 << 16, seed)
    np.testing.assert_array_equal(x1, x0)
    np.testing.assert_array_equal(s1, s0)
    np.testing.assert_array_equal(a1, a0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_four_paths_a_lane_equals_interpreter(eng, name):
    """Specialised kernels with two path pairs a lane (programs that read no
    date behind the frontier; the others keep one pair): per-path payoffs
    and sums bit for bit those of the interpreter, on a ragged path count
    (the last tile pair half empty)."""
    text, tp, spec, notional = CASES[name]
    m, k = eng.model(spec), eng.contract(text, tp)
    n, seed = 4096 + 64 + 37, 0xABD + len(name)
    pc.pc_set_jit(eng.ctx, False)
    x0, s0 = eng.paths(m, k, n, seed)
    a0 = eng.sums(m, k, (1 << 16) + 64 * 3 + 5, seed)
    pc.pc_set_jit(eng.ctx, True)
    try:
        for pairs in (1, 2):
            pc.pc_debug_set_jit_pairs(eng.ctx, pairs)
            x1, s1 = eng.paths(m, k, n, seed)
            a1 = eng.sums(m, k, (1 << 16) + 64 * 3 + 5, seed)
            np.testing.assert_array_equal(x1, x0)
            np.testing.assert_array_equal(s1, s0)
            np.testing.assert_array_equal(a1, a0)
    finally:
        pc.pc_debug_set_jit_pairs(eng.ctx, 0)
        pc.pc_set_jit(eng.ctx, False)


def test_four_paths_a_lane_daily_barrier_full_size(eng):
    """The daily barrier at 2^22 paths with two path pairs a lane: the same
    sums as with one pair and as the interpreter."""
    w = W.daily_barrier()
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    pc.pc_set_jit(eng.ctx, False)
    a0 = eng.sums(m, k, w.n_paths, w.seed)
    pc.pc_set_jit(eng.ctx, True)
    try:
        pc.pc_debug_set_jit_pairs(eng.ctx, 1)
        a1 = eng.sums(m, k, w.n_paths, w.seed)
        pc.pc_debug_set_jit_pairs(eng.ctx, 2)
        a2 = eng.sums(m, k, w.n_paths, w.seed)
    finally:
        pc.pc_debug_set_jit_pairs(eng.ctx, 0)
        pc.pc_set_jit(eng.ctx, False)
    np.testing.assert_array_equal(a1, a0)
    np.testing.assert_array_equal(a2, a0)
    with pytest.raises(pc.PcError):
        pc.pc_debug_set_jit_pairs(eng.ctx, 3)


def test_specialised_matches_oracle_and_is_reused(eng):
    w = W.worst_of_autocall()
    m = eng.model(w.market)
    k = eng.contract(w.il_text, w.tparams)
    pc.pc_set_jit(eng.ctx, True)
    try:
        pc.pc_jit_compile(m, k)
        n, seed = 3000, 77
        x, _ = eng.paths(m, k, n, seed)
        ref, marg = oracle_paths(w.il_text, w.market, w.tparams, n, seed)
        compare(x, ref, marg, w.notional, "specialised autocall")
        # the same program loaded again finds the compiled kernel
        import time
        k2 = eng.contract(w.il_text, w.tparams)
        t = time.perf_counter()
        pc.pc_jit_compile(m, k2)
        assert time.perf_counter() - t < 0.05
        p1 = pc.pc_price(m, k, 1 << 18, 5)
        p2 = pc.pc_price(m, k2, 1 << 18, 5)
        assert p1 == p2
    finally:
        pc.pc_set_jit(eng.ctx, False)
    assert p1 == pc.pc_price(m, k, 1 << 18, 5)


def test_long_program_is_interpreted(eng):
    """A 300-date average (beyond the specialising limit in instructions)
    is interpreted with pc_set_jit on: pc_jit_compile returns at once and
    the price is the interpreter's, bit for bit."""
    days = list(range(1, 301))
    spec = W.MarketSpec([1.0], [0.25], [[1.0]], 0.02, days)
    terms = [f"(model 0 (tplus (tplus 0 $0) {-j}))" for j in range(300)]
    s = terms[0]
    for t_ in terms[1:]:
        s = f"(add {s} {t_})"
    text = f"(mult (max (sub (div {s} 300.0) 1.0) 0.0) (payoff (tplus 0 $0) 0 1))"
    m, k = eng.model(spec), eng.contract(text, [300])
    assert pc.pc_price_info(m, k, 1 << 16).hbm_window == 1
    assert pc.pc_verify_payoff(*pc.pc_assemble(text), [300]).n_insn > pc.JIT_MAX_INSNS
    pc.pc_set_jit(eng.ctx, True)
    try:
        t = time.perf_counter()
        pc.pc_jit_compile(m, k)
        assert time.perf_counter() - t < 0.05
        p1 = pc.pc_price(m, k, 1 << 16, 9)
    finally:
        pc.pc_set_jit(eng.ctx, False)
    assert p1 == pc.pc_price(m, k, 1 << 16, 9)


@pytest.mark.parametrize("gamma", [0, 1])
def test_specialised_control_variate_equals_interpreter(eng, gamma):
    """The run-time specialised control-variate kernel: per-path X, M, M2 and
    the price / pilot sums bit for bit those of the interpreting kernel."""
    w = W.worst_of_autocall()
    m = eng.model(w.market)
    k = eng.contract(w.il_text, w.tparams)
    desc = pc.pc_cv_grid(m, 8, 4.0)
    rng = np.random.default_rng(5)
    tab = torch.tensor((0.3 + 0.4 * rng.standard_normal(pc.pc_cv_table_size(desc))).astype(np.float32),
                       device="cuda")
    for i in range(3):
        desc.delta0[i] = [0.35, 0.25, 0.15][i]
    desc.use_gamma = gamma
    desc.beta, desc.beta2 = 0.9, 0.4
    n, seed = 4096 + 77, 0x5EED0303
    out = {}
    # interpreted; specialised at the default launch bound and at 6 blocks
    for key in ((False, 0), (True, 0), (True, 6)):
        pc.pc_set_jit(eng.ctx, key[0])
        pc.pc_debug_set_cv_min_blocks(eng.ctx, key[1])
        try:
            xm = torch.empty(3 * n, dtype=torch.float32, device="cuda")
            pc.pc_debug_cv_paths(m, k, desc, tab.data_ptr(), n, seed, xm.data_ptr())
            torch.cuda.synchronize()
            res = pc.pc_price_cv(m, k, desc, tab.data_ptr(), 1 << 16, seed)
            betas = pc.pc_cv_beta(m, k, desc, tab.data_ptr(), 1 << 15, seed + 1)
            out[key] = (xm.cpu().numpy(), res, betas)
        finally:
            pc.pc_set_jit(eng.ctx, False)
            pc.pc_debug_set_cv_min_blocks(eng.ctx, 0)
    with pytest.raises(pc.PcError):
        pc.pc_debug_set_cv_min_blocks(eng.ctx, 17)
    for key in ((True, 0), (True, 6)):
        np.testing.assert_array_equal(out[key][0].view(np.uint32), out[(False, 0)][0].view(np.uint32))
        assert out[key][1] == out[(False, 0)][1]
        assert out[key][2] == out[(False, 0)][2]


@pytest.mark.parametrize("name", ["autocall", "lookback", "double_barrier", "nested_loops", "average_40"])
def test_specialised_hbm_window_equals_interpreter(eng, name):
    """Launches whose window of dates lives in HBM (forced, or needed by a
    300-date lookback) run the specialised kernel too: per-path payoffs and
    sums bit for bit those of the interpreting kernel."""
    if name == "average_40":  # 40 dates of a two-asset average, 85 instructions
        w = W.reverse_asian()
        text, tp, spec = W.reverse_asian_text(40), [40], w.market
    else:
        text, tp, spec, _ = CASES[name]
    m, k = eng.model(spec), eng.contract(text, tp)
    pc.pc_set_window_mode(eng.ctx, pc.WINDOW_HBM)
    try:
        assert pc.pc_price_info(m, k, 4096).hbm_window
        n, seed = 4096 + 29, 0x77 + len(name)
        pc.pc_set_jit(eng.ctx, False)
        x0, s0 = eng.paths(m, k, n, seed)
        a0 = eng.sums(m, k, 1 << 15, seed)
        pc.pc_set_jit(eng.ctx, True)
        x1, s1 = eng.paths(m, k, n, seed)
        a1 = eng.sums(m, k, 1 << 15, seed)
    finally:
        pc.pc_set_jit(eng.ctx, False)
        pc.pc_set_window_mode(eng.ctx, pc.WINDOW_AUTO)
    np.testing.assert_array_equal(x1, x0)
    np.testing.assert_array_equal(s1, s0)
    np.testing.assert_array_equal(a1, a0)
