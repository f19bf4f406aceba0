"""GPU pathwise sensitivities (pc_greeks, tangent kernel) against the oracle.

* per path and per underlying: (payoff, d/dS0, d/dsigma) from the kernel
  match the oracle's FP64 pathwise derivative on the same draws, at test
  sizes and, on sampled runs of paths, at the benchmark's size;
* pc_greeks equals the average of the per-path probe;
* European call delta / vega within 3 SE of Black-Scholes;
* pc_greeks agrees with common-random-number bumps of pc_price;
* the torch.autograd.Function returns pc_greeks as gradients;
* the specialised tangent kernel (pc_set_jit) equals the interpreting one,
  bit for bit.
"""
import math

import numpy as np
import pytest

from cases import CASES, SPECS
from gpu_common import Engine, compare, market, tparam_env, torch
import paper_2108_03076_gb300 as pc
import workloads as W
from oracle import closed_forms as cf, il_text, pathwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    yield e
    e.close()


def greek_paths(eng, m, k, n, seed, label, offset=0):
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    x = torch.empty(3 * max(n, 1), dtype=torch.float32, device="cuda")
    pc.pc_debug_greeks_paths(m, k, n, offset, seed, label, out.data_ptr(), x.data_ptr())
    torch.cuda.synchronize()
    g = x[:3 * n].double().cpu().numpy().reshape(n, 3)
    return g[:, 0], g[:, 1], g[:, 2], out.cpu().numpy()


def check_close(got, ref, marg, what, rtol=2e-4):
    """Element-wise within rtol of max(|ref|, 1e-3 * mean |ref|); paths whose
    oracle evaluation compared reals within 1e-5 of a tie, or that straddle a
    kink of max/min within the finite-difference step, may differ: at most
    max(2, 1e-3 N) of them."""
    floor = 1e-3 * np.abs(ref).mean() + 1e-12
    bad = np.abs(got - ref) > rtol * np.maximum(np.abs(ref), floor)
    assert np.all(np.isfinite(got)), what
    n_bad = int(bad.sum())
    assert n_bad <= max(2, 1e-3 * len(ref)), (what, n_bad, np.nonzero(bad)[0][:5])


GREEK_CASES = ["european", "forward", "exchange", "autocall", "autocall_scaled", "worst_knockout",
               "basket_and", "lookback", "nested_loops", "double_barrier"]


@pytest.mark.parametrize("name", GREEK_CASES)
def test_per_path_sensitivities_match_oracle(eng, name):
    text, tp, spec, notional = CASES[name]
    n, seed = 2048 + 11, 0x7777 + len(name)
    m, k = eng.model(spec), eng.contract(text, tp)
    prog = il_text.parse(text)
    for label in range(spec.d):
        v, dS, dv, sums = greek_paths(eng, m, k, n, seed, label)
        x, rS, rv, marg = pathwise.pathwise(prog, market(spec), tparam_env(tp), 0, 1, n, seed, label)
        compare(v, x, marg, notional, (name, label, "value"))
        check_close(dS, rS, marg, (name, label, "delta"))
        check_close(dv, rv, marg, (name, label, "vega"))
        assert sums[6] == n
        assert sums[2] == pytest.approx(dS.sum(), rel=1e-9, abs=1e-9)
        assert sums[4] == pytest.approx(dv.sum(), rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("name", GREEK_CASES)
def test_per_path_tangents_match_oracle_adjoint(eng, name):
    """The tangent kernel's per-path delta and vega against the oracle's
    reverse-mode derivatives (the chain rule, no difference step): the
    price parity's bar, every path within 5e-5 relative except those whose
    decisions were within a tie, at most max(2, 1e-4 N) of them."""
    from test_gpu_adjoint import check_derivative
    text, tp, spec, notional = CASES[name]
    n, seed = 2048 + 11, 0x7777 + len(name)
    m, k = eng.model(spec), eng.contract(text, tp)
    prog = il_text.parse(text)
    x, rS, rv = pathwise.adjoint(prog, market(spec), tparam_env(tp), 0, 1, n, seed)
    _, _, _, marg = pathwise.pathwise(prog, market(spec), tparam_env(tp), 0, 1, n, seed, 0)
    for label in range(spec.d):
        v, dS, dv, _ = greek_paths(eng, m, k, n, seed, label)
        compare(v, x, marg, notional, (name, label, "value"))
        check_derivative(dS, rS[:, label], marg, (name, label, "delta"))
        check_derivative(dv, rv[:, label], marg, (name, label, "vega"))


def test_full_size_sampled_sensitivities(eng):
    """The sensitivities workload at the benchmark's size and seed: per-path
    (payoff, d/dS0, d/dsigma) of every underlying on three runs of paths
    (the first, one in the middle, the ragged end) match the oracle's, and
    the launch's sums are those of all its paths."""
    w = W.GREEKS["greeks_basket_call_3u_5d"]()
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    prog = il_text.parse(w.il_text)
    n = w.n_paths
    mid = int(np.random.default_rng(8).integers(1, n // 512 - 1)) * 512 + 17
    for label in range(w.market.d):
        v, dS, dv, sums = greek_paths(eng, m, k, n, w.seed, label)
        for off in (0, mid, n - 300):
            cnt = min(512, n - off)
            x, rS, rv, marg = pathwise.pathwise(prog, market(w.market), tparam_env(w.tparams), 0, 1, cnt,
                                                w.seed, label, offset=off)
            sl = slice(off, off + cnt)
            compare(v[sl], x, marg, w.notional, ("value", label, off))
            check_close(dS[sl], rS, marg, ("delta", label, off))
            check_close(dv[sl], rv, marg, ("vega", label, off))
        assert sums[6] == n
        assert sums[2] == pytest.approx(dS.sum(), rel=1e-9)
        assert sums[4] == pytest.approx(dv.sum(), rel=1e-9)


@pytest.mark.parametrize("name", sorted(CASES))
def test_specialised_sensitivities_equal_interpreter(eng, name):
    """With pc_set_jit the tangent kernel is specialised to the program: the
    per-path triples and sums of every underlying's launch, and pc_greeks,
    bit for bit those of the interpreting kernel."""
    text, tp, spec, _ = CASES[name]
    n, seed = 4096 + 37, 0x4242 + len(name)
    m, k = eng.model(spec), eng.contract(text, tp)
    got = {}
    for jit in (False, True):
        pc.pc_set_jit(eng.ctx, jit)
        try:
            got[jit] = ([greek_paths(eng, m, k, n, seed, l) for l in range(spec.d)],
                        pc.pc_greeks(m, k, 1 << 15, seed, spec.d))
        finally:
            pc.pc_set_jit(eng.ctx, False)
    (p0, g0), (p1, g1) = got[False], got[True]
    for a, b in zip(p0, p1):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(y, x)
    assert g1[0] == g0[0]
    for x, y in zip(g0[1:], g1[1:]):
        np.testing.assert_array_equal(y, x)


def test_pc_greeks_is_the_mean_of_the_paths(eng):
    text, tp, spec, _ = CASES["autocall_scaled"]
    m, k = eng.model(spec), eng.contract(text, tp)
    n = 30000
    price, delta, vega, se = pc.pc_greeks(m, k, n, 5, spec.d)
    assert price == pytest.approx(pc.pc_price(m, k, n, 5)[0], rel=1e-6)
    for l in range(spec.d):
        v, dS, dv, _ = greek_paths(eng, m, k, n, 5, l)
        assert delta[l] == pytest.approx(dS.mean(), rel=1e-9, abs=1e-12)
        assert vega[l] == pytest.approx(dv.mean(), rel=1e-9, abs=1e-12)
        assert se[1 + l] == pytest.approx(dS.std(ddof=1) / math.sqrt(n), rel=1e-6)


def test_european_greeks_against_black_scholes(eng):
    m = eng.model(SPECS["1u_1d"])
    k = eng.contract(W.european_text(100.0), [1])
    price, delta, vega, se = pc.pc_greeks(m, k, 1 << 22, 0x5EED0001, 1)
    assert abs(price - cf.bs_call(100, 100, 0.03, 0.2, 1.0)) < 3 * se[0]
    assert abs(delta[0] - cf.bs_delta_call(100, 100, 0.03, 0.2, 1.0)) < 3 * se[1]
    assert abs(vega[0] - cf.bs_vega(100, 100, 0.03, 0.2, 1.0)) < 3 * se[2]


# Lipschitz in the path (no payment that jumps when a decision flips), where
# the pathwise derivative is the derivative of the price (reading A16)
WORST_CALL = ("(mult (max (sub (min (div (model 0 12) 100.0) (div (model 1 12) 50.0)) 0.95) 0.0) "
              "(payoff 12 0 1))", [], SPECS["2u_12d"], 1.0)
BUMP_CASES = {"european": CASES["european"], "exchange": CASES["exchange"], "worst_call": WORST_CALL}


@pytest.mark.parametrize("name", list(BUMP_CASES))
def test_greeks_match_common_random_number_bumps(eng, name):
    text, tp, spec, _ = BUMP_CASES[name]
    k = eng.contract(text, tp)
    n, seed, h = 1 << 20, 99, 1e-4
    price, delta, vega, se = pc.pc_greeks(eng.model(spec), k, n, seed, spec.d)
    for l in range(spec.d):
        for field, got, scale in (("S0", delta[l], se[1 + l]), ("sigma", vega[l], se[1 + spec.d + l])):
            vals = []
            for sgn in (+1, -1):
                s = W.MarketSpec(**{**vars(spec)})
                arr = list(getattr(s, field))
                step = h * arr[l]
                arr[l] += sgn * step
                setattr(s, field, arr)
                vals.append(pc.pc_price(eng.model(s), k, n, seed)[0])
            fd = (vals[0] - vals[1]) / (2 * step)
            assert abs(fd - got) <= 2e-3 * abs(got) + 0.2 * scale + 1e-6, (name, l, field, fd, got)


def test_autograd_function_returns_pathwise_gradients(eng):
    from paper_2108_03076_gb300.autograd import mc_price
    text, tp, spec, _ = CASES["exchange"]
    k = eng.contract(text, tp)
    S0 = torch.tensor(spec.S0, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(spec.sigma, dtype=torch.float64, requires_grad=True)
    p = mc_price(eng.ctx, k, S0, sig, spec.corr, spec.r, spec.days, 1 << 18, 4)
    gS, gv = torch.autograd.grad(2.0 * p, [S0, sig])
    m = eng.model(spec)
    price, delta, vega, _ = pc.pc_greeks(m, k, 1 << 18, 4, spec.d)
    assert float(p.detach()) == pytest.approx(price, rel=1e-12)
    np.testing.assert_allclose(gS.numpy(), 2.0 * delta, rtol=1e-12)
    np.testing.assert_allclose(gv.numpy(), 2.0 * vega, rtol=1e-12)
