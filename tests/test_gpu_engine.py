"""GPU parity of the fused pricing kernel against the FP64 oracle.

* Philox4x32-10 integers: bit-exact against the oracle and cuRAND's device
  function;
* simulated path values against the oracle's generator;
* per-path discounted payoffs on identical draws for every workload and for
  stress programs (nested loopif, lookback, history, now/texpr, parties),
  at sizes spanning many tiles with a ragged tail, counters crossing 2^32;
* full-size workloads in the launch configuration the benchmark times, on
  sampled paths the oracle computes one by one (the window of dates in HBM
  for the 300-date average), and the specialised kernel the benchmark
  runs equal to the interpreter there, bit for bit;
* prices against closed forms; edge cases and error statuses.
"""
import math

import numpy as np
import pytest

from gpu_common import Engine, compare, curand_reference_lib, market, oracle_paths, torch
import paper_2108_03076_gb300 as pc
import workloads as W
from oracle import closed_forms as cf, paths as opaths
from cases import CASES, SPECS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    yield e
    e.close()


# ---------------------------------------------------------------------------
# Philox
# ---------------------------------------------------------------------------


def test_philox_bit_exact_against_oracle_and_curand(eng):
    rng = np.random.default_rng(11)
    n = 1 << 16
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:8] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
               [2 ** 32 - 1] * 4, [5, 2 ** 31, 7, 2 ** 32 - 2], [3, 3, 3, 3]]
    for key in [(0, 0), (0x5EED0001, 0), (0xDEADBEEF, 0x0BADF00D), (2 ** 32 - 1, 2 ** 32 - 1)]:
        d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
        d_out = torch.zeros_like(d_ctr)
        pc.pc_debug_philox(eng.ctx, d_ctr.data_ptr(), key[0], key[1], d_out.data_ptr(), n)
        got = d_out.cpu().numpy().view(np.uint32)
        want = np.stack([v.astype(np.uint32) for v in opaths.philox4x32_10(
            [ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3]], key)], axis=1)
        np.testing.assert_array_equal(got, want)
        L = curand_reference_lib()
        d_ref = torch.zeros_like(d_ctr)
        assert L.curand_philox_ref(d_ctr.data_ptr(), key[0], key[1], d_ref.data_ptr(), n) == 0
        np.testing.assert_array_equal(d_ref.cpu().numpy().view(np.uint32), want)


# ---------------------------------------------------------------------------
# Path generator
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(SPECS))
def test_paths_match_oracle(eng, name):
    spec = SPECS[name]
    n, seed, off, stream = 1000, 0x1234567, (1 << 32) - 300, 7
    m = eng.model(spec)
    S = torch.zeros(n * spec.d * (spec.n + 1), dtype=torch.float32, device="cuda")
    pc.pc_debug_paths(m, n, off, seed, stream, S.data_ptr())
    got = S.cpu().numpy().astype(np.float64).reshape(n, spec.d, spec.n + 1)
    want = opaths.simulate(market(spec), seed, stream, np.arange(off, off + n, dtype=np.uint64))
    rel = np.abs(got - want) / want
    assert rel.max() < 2e-5, rel.max()


# ---------------------------------------------------------------------------
# Per-path parity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(CASES))
def test_per_path_parity(eng, name):
    text, tp, spec, notional = CASES[name]
    n = 4096 + 37
    for off, stream in [(0, 0), ((1 << 32) - 1000, 5)]:
        m, k = eng.model(spec), eng.contract(text, tp)
        x, sums = eng.paths(m, k, n, 0xABCDEF + len(name), off, stream)
        ref, marg = oracle_paths(text, spec, tp, n, 0xABCDEF + len(name), off, stream)
        compare(x, ref, marg, notional, name)
        assert sums[2] == n
        assert sums[0] == pytest.approx(x.sum(), rel=1e-12, abs=1e-9)
        assert sums[1] == pytest.approx((x * x).sum(), rel=1e-12, abs=1e-9)


def test_party_folding_signs(eng):
    text, tp, spec, _ = CASES["european"]
    m = eng.model(spec)
    k01, k10, k02 = eng.contract(text, tp, 0, 1), eng.contract(text, tp, 1, 0), eng.contract(text, tp, 0, 2)
    x01, _ = eng.paths(m, k01, 500, 9)
    x10, _ = eng.paths(m, k10, 500, 9)
    x02, _ = eng.paths(m, k02, 500, 9)
    np.testing.assert_array_equal(x10, -x01)
    assert np.all(x02 == 0.0)


# ---------------------------------------------------------------------------
# Full-size workloads, sampled paths, benchmark launch configuration
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("wl", ["european_call_1u_1d", "worst_of_autocall_3u_5d", "daily_barrier_3u_365d",
                                "reverse_asian_2u_300d"])
def test_full_size_sampled_parity(eng, wl):
    w = W.ALL[wl]()
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    x, sums = eng.paths(m, k, w.n_paths, w.seed)
    plain = eng.sums(m, k, w.n_paths, w.seed)           # the benchmark's kernel
    assert plain[0] == sums[0] and plain[1] == sums[1] and plain[2] == w.n_paths
    assert sums[0] == pytest.approx(x.sum(), rel=1e-10)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.integers(0, w.n_paths, 1500), np.arange(w.n_paths - 40, w.n_paths)]))
    ref, marg = oracle_paths(w.il_text, w.market, w.tparams, 0, w.seed, paths=idx.astype(np.uint64))
    compare(x[idx], ref, marg, w.notional, wl)


@pytest.mark.parametrize("wl", ["worst_of_autocall_3u_5d", "daily_barrier_3u_365d"])
def test_full_size_specialised_kernel_equals_interpreter(eng, wl):
    """The benchmark's default kernel (specialised to the program) at the
    benchmark's size and seed: the interpreter's sums and per-path payoffs,
    bit for bit (so the sampled oracle parity above carries over)."""
    w = W.ALL[wl]()
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    x0, s0 = eng.paths(m, k, w.n_paths, w.seed)
    pc.pc_set_jit(eng.ctx, True)
    try:
        x1, s1 = eng.paths(m, k, w.n_paths, w.seed)
        plain = eng.sums(m, k, w.n_paths, w.seed)
    finally:
        pc.pc_set_jit(eng.ctx, False)
    np.testing.assert_array_equal(x1, x0)
    np.testing.assert_array_equal(s1, s0)
    np.testing.assert_array_equal(plain, s0)


# ---------------------------------------------------------------------------
# Prices
# ---------------------------------------------------------------------------


def test_prices_against_closed_forms(eng):
    mk = SPECS["1u_1d"]
    m = eng.model(mk)
    n = 1 << 22
    for text, want in [(W.european_text(100.0), cf.bs_call(100, 100, 0.03, 0.2, 1.0)),
                       (W.digital_text(100.0), cf.digital_call(100, 100, 0.03, 0.2, 1.0)),
                       (W.forward_text(100.0), cf.forward(100, 100, 0.03, 1.0))]:
        p, se = pc.pc_price(m, eng.contract(text, [1]), n, 0x5EED0001)
        assert abs(p - want) < 3 * se, (text, p, want, se)
    p, se = pc.pc_price(m, eng.contract(W.zero_coupon_text(), [1]), n, 1)
    assert p == pytest.approx(math.exp(-0.03), rel=1e-7) and se < 1e-6
    # C1 at its configured 2^16 paths
    w = W.european_call()
    p, se = pc.pc_price(m, eng.contract(w.il_text, w.tparams), w.n_paths, w.seed)
    assert abs(p - 9.413403383853016) < 3 * se and se / p == pytest.approx(0.00586, rel=0.05)
    # exchange option, 2 correlated assets (Margrabe)
    mk2 = W.MarketSpec([100.0, 95.0], [0.25, 0.3], W.const_corr(2, 0.5), 0.03, [182, 365])
    p, se = pc.pc_price(eng.model(mk2), eng.contract(W.exchange_text(), [2]), n, 3)
    assert abs(p - cf.margrabe(100, 95, 0.25, 0.3, 0.5, 1.0)) < 3 * se


def test_gpu_price_matches_oracle_estimate_autocall(eng):
    """pc_price == mean of the kernel's own per-path values; those match the
    oracle path by path, so the price matches the oracle's estimate up to
    the per-path tolerance and the few decisions taken at a tie."""
    w = W.worst_of_autocall()
    n = 1 << 16
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    p, se = pc.pc_price(m, k, n, w.seed)
    x, _ = eng.paths(m, k, n, w.seed)
    ref, marg = oracle_paths(w.il_text, w.market, w.tparams, n, w.seed)
    flips = compare(x, ref, marg, w.notional)
    assert p == pytest.approx(x.mean(), rel=1e-12)
    assert se == pytest.approx(x.std(ddof=1) / math.sqrt(n), rel=1e-9)
    assert abs(p - ref.mean()) <= 1e-5 * np.maximum(np.abs(ref), 1.0).mean() + 2.0 * flips / n


# ---------------------------------------------------------------------------
# Edge cases and errors
# ---------------------------------------------------------------------------


def test_edge_sizes_offsets_determinism(eng):
    text, tp, spec, notional = CASES["autocall"]
    m, k = eng.model(spec), eng.contract(text, tp)
    for n in [1, 2, 31, 63, 64, 65, 127, 129]:
        x, sums = eng.paths(m, k, n, 77, 3)
        ref, marg = oracle_paths(text, spec, tp, n, 77, 3)
        compare(x, ref, marg, notional)
        assert sums[2] == n
    # disjoint ranges compose; per-path values do not depend on the launch
    a = eng.sums(m, k, 10000, 5, 0)
    b = eng.sums(m, k, 7000, 5, 0) + eng.sums(m, k, 3000, 5, 7000)
    assert a[0] == pytest.approx(b[0], rel=1e-12) and a[1] == pytest.approx(b[1], rel=1e-12)
    x1, _ = eng.paths(m, k, 10000, 5)
    x2, _ = eng.paths(m, k, 3000, 5, 7000)
    np.testing.assert_array_equal(x1[7000:], x2)
    # deterministic
    assert pc.pc_price(m, k, 100000, 8) == pc.pc_price(m, k, 100000, 8)
    # different streams give different draws
    assert eng.sums(m, k, 1000, 8, 0, 0)[0] != eng.sums(m, k, 1000, 8, 0, 1)[0]


def expect_error(status, fn, *a):
    with pytest.raises(pc.PcError) as ei:
        fn(*a)
    assert ei.value.name == status, str(ei.value)


def test_error_statuses(eng):
    m12 = eng.model(SPECS["2u_12d"])
    expect_error("PC_ERANGE", pc.pc_price, m12, eng.contract("(mult (model 0 13) (payoff 1 0 1))"), 100, 1)
    expect_error("PC_ERANGE", pc.pc_price, m12, eng.contract("(mult (model 2 1) (payoff 1 0 1))"), 100, 1)
    expect_error("PC_ERANGE", pc.pc_price, m12, eng.contract("(mult (model 0 -1) (payoff 1 0 1))"), 100, 1)
    expect_error("PC_ERANGE", pc.pc_price, m12, eng.contract("(payoff 13 0 1)"), 100, 1)
    m400 = eng.model(W.MarketSpec([1.0], [0.2], [[1.0]], 0.0, list(range(1, 401))))
    far = eng.contract("(add (model 0 301) (model 0 1))")
    pc.pc_set_window_mode(eng.ctx, pc.WINDOW_SHARED)      # lookback 300: shared windows keep 256
    try:
        expect_error("PC_ERANGE", pc.pc_price, m400, far, 100, 1)
        pc.pc_price(m400, eng.contract("(add (model 0 201) (model 0 1))"), 100, 1)   # lookback 200 fits
    finally:
        pc.pc_set_window_mode(eng.ctx, pc.WINDOW_AUTO)
    pc.pc_price(m400, far, 100, 1)                         # the HBM window holds it
    expect_error("PC_EINVAL", pc.pc_price, m12, eng.contract("(model 0 1)"), 1, 1)
    expect_error("PC_ENOTPD", pc.pc_model_create, eng.ctx, [1.0, 1.0], [0.2, 0.2],
                 [[1.0, 1.0], [1.0, 1.0]], 0.0, [1])
    expect_error("PC_EINVAL", pc.pc_model_create, eng.ctx, [1.0], [0.2], [[1.0]], 0.0, [2, 2])
    expect_error("PC_ELIMIT", pc.pc_model_create, eng.ctx, [1.0] * 5, [0.2] * 5,
                 np.eye(5).tolist(), 0.0, [1])
    w, k = pc.pc_assemble("(model 0 1)")
    expect_error("PC_EBYTECODE", pc.pc_load_payoff, eng.ctx, w[:1], k, (), 0, 1)
    # the context is still usable after the errors
    p, se = pc.pc_price(m12, eng.contract("(mult (model 0 12) (payoff 12 0 1))"), 1000, 1)
    assert math.isfinite(p) and se > 0
