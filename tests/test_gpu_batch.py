"""GPU portfolio pricing (pc_batch_* / pc_price_batch).

* Every contract of a batch gets exactly the sums (bit for bit) of a
  single-contract launch with Philox stream word = its index, for mixed
  underlying counts, program shapes, date grids and ragged path budgets,
  under every launch shape and after the autotuner;
* the 1024-contract portfolio: sampled contracts bit-identical to their
  single launches, and short-dated sampled contracts against the oracle's
  FP64 payoffs on the same draws;
* argument errors come back as status codes.
"""
import numpy as np
import pytest

from cases import CASES
from gpu_common import Engine, TIE, market, tparam_env, torch
import paper_2108_03076_gb300 as pc
import workloads as W
from oracle import il_text, mc

pytestmark = pytest.mark.gpu

SEED = 0x5EED0004
BUDGETS = [2, 63, 64, 65, 1000, 4097, 12345, 777, 64 * 300 + 5, 129]


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    yield e
    e.close()


@pytest.fixture(scope="module")
def mixed(eng):
    """Test cases plus the first 40 portfolio contracts, ragged budgets."""
    models, contracts = [], []
    for name in sorted(CASES):
        text, tp, spec, _ = CASES[name]
        models.append(eng.model(spec))
        contracts.append(eng.contract(text, tp))
    for it in W.portfolio()[:40]:
        models.append(eng.model(it.market))
        contracts.append(eng.contract(it.il_text, it.tparams))
    n_paths = [BUDGETS[i % len(BUDGETS)] for i in range(len(contracts))]
    return models, contracts, n_paths


def single_sums(eng, models, contracts, n_paths, idx):
    return np.array([eng.sums(models[i], contracts[i], n_paths[i], SEED, 0, i)[:3] for i in idx])


def check_identical(eng, plan, models, contracts, n_paths, want=None):
    pc.pc_batch_launch(plan)
    price, se, sums = pc.pc_batch_results(plan, len(contracts), sums=True)
    if want is None:
        want = single_sums(eng, models, contracts, n_paths, range(len(contracts)))
    np.testing.assert_array_equal(sums, want)
    N = np.asarray(n_paths, dtype=np.float64)
    np.testing.assert_array_equal(price, want[:, 0] / N)
    return want, price, se


def test_batch_is_bit_identical_to_single_launches(eng, mixed):
    models, contracts, n_paths = mixed
    plan = pc.pc_batch_create(models, contracts, n_paths, SEED)
    try:
        info = pc.pc_batch_query(plan)
        assert info.n_contracts == len(contracts)
        assert info.n_tiles == sum((n + 63) // 64 for n in n_paths)
        assert info.n_groups >= 4 and info.n_units >= info.n_groups
        want, price, se = check_identical(eng, plan, models, contracts, n_paths)
        # a second replay of the graph gives the same bits
        _, price2, se2 = check_identical(eng, plan, models, contracts, n_paths, want)
        np.testing.assert_array_equal(price, price2)
        np.testing.assert_array_equal(se, se2)
        p1, s1 = pc.pc_price_batch(models, contracts, n_paths, SEED)
        np.testing.assert_array_equal(p1, price)
        np.testing.assert_array_equal(s1, se)
    finally:
        pc.pc_batch_destroy(plan)


@pytest.mark.parametrize("block,split", [(32, 1), (64, 8), (128, 128), (128, 1000)])
def test_every_launch_shape_gives_the_same_bits(eng, mixed, block, split):
    models, contracts, n_paths = mixed
    want = single_sums(eng, models, contracts, n_paths, range(len(contracts)))
    plan = pc.pc_batch_create(models, contracts, n_paths, SEED, block=block, unit_split=split)
    try:
        info = pc.pc_batch_query(plan)
        assert (info.config.block, info.config.unit_split) == (block, split)
        check_identical(eng, plan, models, contracts, n_paths, want)
    finally:
        pc.pc_batch_destroy(plan)


def test_autotuner_keeps_results_and_reports_its_choice(eng, mixed):
    models, contracts, n_paths = mixed
    want = single_sums(eng, models, contracts, n_paths, range(len(contracts)))
    plan = pc.pc_batch_create(models, contracts, n_paths, SEED)
    try:
        pc.pc_batch_tune(plan, 1)
        info = pc.pc_batch_query(plan)
        assert info.tuned == 1 and info.last_ms > 0
        assert info.config.block in (64, 128) and info.config.unit_split in (8, 32, 128)
        assert info.paths_per_thread >= 2
        check_identical(eng, plan, models, contracts, n_paths, want)
    finally:
        pc.pc_batch_destroy(plan)


@pytest.mark.parametrize("block,split", [(128, 128), (64, 8)])
def test_single_launch_gives_the_same_bits(eng, mixed, block, split):
    """One launch of the kernel for every underlying count (the contracts'
    generators selected per unit) against single-contract launches, and
    back to the grouped arrangement."""
    models, contracts, n_paths = mixed
    want = single_sums(eng, models, contracts, n_paths, range(len(contracts)))
    plan = pc.pc_batch_create(models, contracts, n_paths, SEED, block=block, unit_split=split)
    try:
        grouped = pc.pc_batch_query(plan).n_groups
        pc.pc_batch_set_single_launch(plan, True)
        assert pc.pc_batch_query(plan).n_groups == 1
        check_identical(eng, plan, models, contracts, n_paths, want)
        pc.pc_batch_tune(plan, 1)
        check_identical(eng, plan, models, contracts, n_paths, want)
        pc.pc_batch_set_single_launch(plan, False)
        assert pc.pc_batch_query(plan).n_groups == grouped
        check_identical(eng, plan, models, contracts, n_paths, want)
        with pytest.raises(pc.PcError):   # only 0 and 1
            pc._check(pc.lib().pc_batch_set_single_launch(pc.VP(plan), 2))
    finally:
        pc.pc_batch_destroy(plan)


@pytest.fixture(scope="module")
def portfolio(eng):
    items = W.portfolio()
    models = [eng.model(it.market) for it in items]
    contracts = [eng.contract(it.il_text, it.tparams) for it in items]
    return items, models, contracts


def test_full_portfolio_sampled_parity(eng, portfolio):
    items, models, contracts = portfolio
    n_paths = [it.n_paths for it in items]
    plan = pc.pc_batch_create(models, contracts, n_paths, SEED)
    try:
        pc.pc_batch_tune(plan, 1)
        pc.pc_batch_launch(plan)
        price, se, sums = pc.pc_batch_results(plan, len(items), sums=True)
    finally:
        pc.pc_batch_destroy(plan)
    assert np.all(np.isfinite(price)) and np.all(se >= 0)
    rng = np.random.default_rng(3)
    idx = sorted(rng.choice(len(items), 24, replace=False))
    np.testing.assert_array_equal(sums[idx], single_sums(eng, models, contracts, n_paths, idx))
    # oracle on identical draws, one short contract of each template
    seen = set()
    for i, it in enumerate(items):
        if it.template in seen or it.market.n > 24 or it.n_paths > 20000:
            continue
        seen.add(it.template)
        x, marg = mc.payoffs(il_text.parse(it.il_text), market(it.market), tparam_env(it.tparams),
                             0, 1, it.n_paths, SEED, i, 0, with_margins=True)
        n = it.n_paths
        ties = int((marg < TIE).sum())
        tol = 1e-5 * np.abs(x).mean() + (ties + 2) * np.abs(x).max() / n + 1e-12
        assert abs(price[i] - x.mean()) <= tol, (i, it.template, price[i], x.mean(), ties)
        assert sums[i, 2] == n
    assert len(seen) >= 4, seen


def test_argument_errors(eng, mixed):
    models, contracts, n_paths = mixed
    with pytest.raises(pc.PcError) as e:
        pc.pc_batch_create([], [], [], SEED)
    assert e.value.name == "PC_EINVAL"
    with pytest.raises(pc.PcError) as e:
        pc.pc_batch_create(models[:2], contracts[:2], [100, 1], SEED)
    assert e.value.name == "PC_EINVAL"
    with pytest.raises(pc.PcError) as e:
        pc.pc_batch_create(models[:1], contracts[:1], [100], SEED, block=96)
    assert e.value.name == "PC_EINVAL"
    # a program reading underlying 1 on a one-underlying model
    m1 = eng.model(W.MarketSpec([1.0], [0.2], [[1.0]], 0.0, [10, 20]))
    k2 = eng.contract("(mult (model 1 2) (payoff 2 0 1))")
    with pytest.raises(pc.PcError) as e:
        pc.pc_batch_create([m1], [k2], [100], SEED)
    assert e.value.name == "PC_ERANGE"
    plan = pc.pc_batch_create(models[:3], contracts[:3], [100, 200, 300], SEED)
    try:
        with pytest.raises(pc.PcError) as e:
            pc.pc_batch_results(plan, 3)
        assert e.value.name == "PC_EINVAL"
        pc.pc_batch_launch(plan)
        p, s = pc.pc_batch_results(plan, 3)
        assert np.all(np.isfinite(p))
    finally:
        pc.pc_batch_destroy(plan)


def test_programs_loaded_in_one_call_price_the_same(eng, mixed):
    """pc_load_payoffs: the test programs and 40 portfolio contracts loaded
    in one call price bit for bit as the ones loaded one at a time (one-shot
    pc_price_batch, no graph); a bad program names its index and leaves
    nothing loaded."""
    models, contracts, n_paths = mixed
    progs = []
    for name in sorted(CASES):
        text, tp, spec, _ = CASES[name]
        w, k = pc.pc_assemble(text)
        progs.append((w, k, tp))
    for it in W.portfolio()[:40]:
        w, k = pc.pc_assemble(it.il_text)
        progs.append((w, k, it.tparams))
    ks = pc.pc_load_payoffs(eng.ctx, progs)
    try:
        assert len(ks) == len(contracts)
        p1, s1 = pc.pc_price_batch(models, ks, n_paths, SEED)
        p0, s0 = pc.pc_price_batch(models, contracts, n_paths, SEED)
        np.testing.assert_array_equal(p1, p0)
        np.testing.assert_array_equal(s1, s0)
    finally:
        for k in ks:
            pc.pc_contract_destroy(k)
    bad = list(progs[:5])
    bad[3] = (np.asarray(bad[3][0], np.uint32)[:-1], bad[3][1], bad[3][2])  # truncated bytecode
    with pytest.raises(pc.PcError) as e:
        pc.pc_load_payoffs(eng.ctx, bad)
    assert "program 3" in str(e.value)


def test_specialised_contracts_in_the_plan_give_the_same_bits(eng, mixed):
    """With pc_set_jit the costliest contracts run on their own specialised
    kernels inside the replay: the same bits as single launches, and on the
    1024-contract portfolio the same prices as the all-interpreted plan
    (one-shot pricing too)."""
    models, contracts, n_paths = mixed
    pc.pc_set_jit(eng.ctx, True)
    try:
        plan = pc.pc_batch_create(models, contracts, n_paths, SEED)
        try:
            assert pc.pc_batch_query(plan).n_specialised >= 1
            check_identical(eng, plan, models, contracts, n_paths)
        finally:
            pc.pc_batch_destroy(plan)
    finally:
        pc.pc_set_jit(eng.ctx, False)
    items = W.portfolio()
    pm = [eng.model(it.market) for it in items]
    pk = [eng.contract(it.il_text, it.tparams) for it in items]
    pn = [it.n_paths for it in items]
    p0, s0 = pc.pc_price_batch(pm, pk, pn, SEED)
    pc.pc_set_jit(eng.ctx, True)
    try:
        plan = pc.pc_batch_create(pm, pk, pn, SEED)
        try:
            assert pc.pc_batch_query(plan).n_specialised > 8
            pc.pc_batch_launch(plan)
            p1, s1 = pc.pc_batch_results(plan, len(items))
        finally:
            pc.pc_batch_destroy(plan)
        p2, s2 = pc.pc_price_batch(pm, pk, pn, SEED)
    finally:
        pc.pc_set_jit(eng.ctx, False)
    np.testing.assert_array_equal(p1, p0)
    np.testing.assert_array_equal(s1, s0)
    np.testing.assert_array_equal(p2, p0)
