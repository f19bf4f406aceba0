"""GPU adjoint sensitivities (pc_greeks_adjoint) against the oracle.

* per path: (payoff, d/dS0_l, d/dsigma_l for every l) from one adjoint
  launch match the oracle's reverse-mode derivative (oracle.pathwise.adjoint,
  pinned against closed forms and central differences) on the same draws;
* the launch's sums are those of its paths, and pc_greeks_adjoint their
  means;
* per path, the adjoint equals the tangent kernel's derivatives (two
  independent device computations);
* European call delta and vega within 3 SE of Black-Scholes.
"""
import math

import numpy as np
import pytest

from cases import CASES, SPECS
from gpu_common import TIE, Engine, compare, market, tparam_env, torch
import paper_2108_03076_gb300 as pc
import workloads as W
from oracle import closed_forms as cf, il_text, pathwise

pytestmark = pytest.mark.gpu

GREEK_CASES = ["european", "forward", "exchange", "autocall", "autocall_scaled", "worst_knockout",
               "basket_and", "lookback", "nested_loops", "double_barrier"]


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    yield e
    e.close()


def adjoint_paths(m, k, n, seed, d, offset=0):
    """(x [n], dS [n, d], dv [n, d], sums [2 (1 + 2d) + 1])."""
    v = 1 + 2 * d
    out = torch.zeros(2 * v + 1, dtype=torch.float64, device="cuda")
    x = torch.full((v * max(n, 1),), float("nan"), dtype=torch.float32, device="cuda")
    pc.pc_debug_adjoint_paths(m, k, n, offset, seed, out.data_ptr(), x.data_ptr())
    torch.cuda.synchronize()
    g = x[:v * n].double().cpu().numpy().reshape(n, v)
    return g[:, 0], g[:, 1:1 + d], g[:, 1 + d:], out.cpu().numpy()


def check_derivative(got, ref, marg, what, rtol=5e-5):
    """|got - ref| <= rtol max(|ref|, 0.25 mean |ref|) on every path whose
    decisions were not within TIE of a tie; the others may take the other
    branch in FP32 on at most max(2, 1e-4 N) paths.  The floor: a vega term
    S (X - sigma tau) carries FP32's absolute error in X (about 5e-7 from the
    normals) times S, which is of the order of the mean |vega| when X -
    sigma tau is small."""
    assert np.all(np.isfinite(got)), what
    floor = 0.25 * np.abs(ref).mean() + 1e-12
    bad = np.abs(got - ref) > rtol * np.maximum(np.abs(ref), floor)
    amb = marg < TIE
    hard = np.nonzero(bad & ~amb)[0]
    assert len(hard) == 0, (what, hard[:5], got[hard[:5]], ref[hard[:5]])
    assert int((bad & amb).sum()) <= max(2, 1e-4 * len(ref)), what


@pytest.mark.parametrize("name", GREEK_CASES)
def test_per_path_adjoint_matches_oracle_adjoint(eng, name):
    text, tp, spec, notional = CASES[name]
    n, seed = 2048 + 11, 0x7777 + len(name)
    m, k = eng.model(spec), eng.contract(text, tp)
    v, dS, dv, sums = adjoint_paths(m, k, n, seed, spec.d)
    prog = il_text.parse(text)
    x, rS, rv = pathwise.adjoint(prog, market(spec), tparam_env(tp), 0, 1, n, seed)
    _, _, _, marg = pathwise.pathwise(prog, market(spec), tparam_env(tp), 0, 1, n, seed, 0)
    compare(v, x, marg, notional, (name, "value"))
    for l in range(spec.d):
        check_derivative(dS[:, l], rS[:, l], marg, (name, l, "delta"))
        check_derivative(dv[:, l], rv[:, l], marg, (name, l, "vega"))
    assert sums[-1] == n
    q = np.concatenate([v[:, None], dS, dv], axis=1)
    for j in range(q.shape[1]):
        assert sums[2 * j] == pytest.approx(q[:, j].sum(), rel=1e-9, abs=1e-9)
        assert sums[2 * j + 1] == pytest.approx((q[:, j] ** 2).sum(), rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("name", ["exchange", "autocall_scaled", "basket_and", "double_barrier"])
def test_adjoint_equals_tangent_kernel(eng, name):
    """Two device computations of the same derivatives: reverse mode (one
    launch, all underlyings) and tangent mode (one launch per underlying)."""
    from test_gpu_greeks import greek_paths
    text, tp, spec, _ = CASES[name]
    n, seed = 4096 + 5, 0x51 + len(name)
    m, k = eng.model(spec), eng.contract(text, tp)
    v, dS, dv, _ = adjoint_paths(m, k, n, seed, spec.d)
    _, _, _, marg = pathwise.pathwise(il_text.parse(text), market(spec), tparam_env(tp), 0, 1, n, seed, 0)
    for l in range(spec.d):
        tv, tS, tvv, _ = greek_paths(eng, m, k, n, seed, l)
        np.testing.assert_array_equal(v, tv)
        check_derivative(dS[:, l], tS, marg, (name, l, "delta"))
        check_derivative(dv[:, l], tvv, marg, (name, l, "vega"))


def test_pc_greeks_adjoint_is_the_mean_of_the_paths(eng):
    text, tp, spec, _ = CASES["autocall_scaled"]
    m, k = eng.model(spec), eng.contract(text, tp)
    n = 30000
    price, delta, vega, se = pc.pc_greeks_adjoint(m, k, n, 5, spec.d)
    assert price == pytest.approx(pc.pc_price(m, k, n, 5)[0], rel=1e-6)
    v, dS, dv, _ = adjoint_paths(m, k, n, 5, spec.d)
    for l in range(spec.d):
        assert delta[l] == pytest.approx(dS[:, l].mean(), rel=1e-9, abs=1e-12)
        assert vega[l] == pytest.approx(dv[:, l].mean(), rel=1e-9, abs=1e-12)
        assert se[1 + l] == pytest.approx(dS[:, l].std(ddof=1) / math.sqrt(n), rel=1e-6)


def test_european_adjoint_against_black_scholes(eng):
    m = eng.model(SPECS["1u_1d"])
    k = eng.contract(W.european_text(100.0), [1])
    price, delta, vega, se = pc.pc_greeks_adjoint(m, k, 1 << 22, 0x5EED0001, 1)
    assert abs(price - cf.bs_call(100, 100, 0.03, 0.2, 1.0)) < 3 * se[0]
    assert abs(delta[0] - cf.bs_delta_call(100, 100, 0.03, 0.2, 1.0)) < 3 * se[1]
    assert abs(vega[0] - cf.bs_vega(100, 100, 0.03, 0.2, 1.0)) < 3 * se[2]


def test_full_size_sampled_adjoint(eng):
    """The sensitivities workload at the benchmark's size and seed: the
    launch's per-path values on three runs of paths (the first, one in the
    middle, the ragged end) match the oracle's adjoint."""
    w = W.GREEKS["greeks_basket_call_3u_5d"]()
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    prog = il_text.parse(w.il_text)
    n = w.n_paths
    v, dS, dv, sums = adjoint_paths(m, k, n, w.seed, w.market.d)
    mid = int(np.random.default_rng(8).integers(1, n // 512 - 1)) * 512 + 17
    for off in (0, mid, n - 300):
        cnt = min(512, n - off)
        x, rS, rv = pathwise.adjoint(prog, market(w.market), tparam_env(w.tparams), 0, 1, cnt, w.seed,
                                     offset=off)
        _, _, _, marg = pathwise.pathwise(prog, market(w.market), tparam_env(w.tparams), 0, 1, cnt,
                                          w.seed, 0, offset=off)
        sl = slice(off, off + cnt)
        compare(v[sl], x, marg, w.notional, ("value", off))
        for l in range(w.market.d):
            check_derivative(dS[sl, l], rS[:, l], marg, ("delta", l, off))
            check_derivative(dv[sl, l], rv[:, l], marg, ("vega", l, off))
    assert sums[-1] == n


@pytest.mark.parametrize("name", GREEK_CASES)
def test_specialised_adjoint_equals_interpreter(eng, name):
    """The adjoint kernel compiled at run time for the program (pc_set_jit):
    per-path value, deltas and vegas and the launch's sums bit for bit those
    of the interpreting adjoint kernel (programs with many reading
    instructions stay interpreted)."""
    text, tp, spec, _ = CASES[name]
    n, seed = 4096 + 21, 0x61 + len(name)
    m, k = eng.model(spec), eng.contract(text, tp)
    ref = adjoint_paths(m, k, n, seed, spec.d)
    pc.pc_set_jit(eng.ctx, True)
    try:
        got = adjoint_paths(m, k, n, seed, spec.d)
    finally:
        pc.pc_set_jit(eng.ctx, False)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


def test_specialised_adjoint_full_size():
    """The sensitivities workload of 4 underlyings and 365 dates at 2^20
    paths: the specialised adjoint's sums equal the interpreter's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    try:
        w = W.GREEKS["greeks_daily_barrier_4u_365d"]()
        m, k = e.model(w.market), e.contract(w.il_text, w.tparams)
        outs = []
        for jit in (False, True):
            pc.pc_set_jit(e.ctx, jit)
            out = torch.zeros(2 * (1 + 2 * w.market.d) + 1, dtype=torch.float64, device="cuda")
            pc.pc_greeks_adjoint_async(m, k, w.n_paths, 0, w.seed, 0, out.data_ptr())
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        pc.pc_set_jit(e.ctx, False)
        np.testing.assert_array_equal(outs[1], outs[0])
    finally:
        e.close()
