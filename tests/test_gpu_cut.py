"""One compiled contract priced at several valuation times (Sec. 4.1,
"avoiding recompilation"): the worst-of autocallable is put through
pc_cut_payoff and loaded once; each model then places the valuation date
at IL time now = 0..4 (the dates before now become history, the spot is
the realised value at now).  Per path the kernel matches the oracle's
evaluation of its own cutPayoff of the contract at that now (Theorem 5:
the value of the cashflows from now on); at now = 0 the cut program gives
the uncut program's payoffs bit for bit."""
import numpy as np
import pytest

from gpu_common import Engine, compare, oracle_paths, torch
import paper_2108_03076_gb300 as pc
import workloads as W
from oracle import il, il_text

pytestmark = pytest.mark.gpu

# realised worst-of path of the three underlyings at IL times 0..5 (annual)
REALISED = np.array([[1.0, 1.0, 1.0], [1.04, 0.97, 1.01], [0.95, 0.99, 1.06], [1.08, 0.62, 0.9],
                     [1.1, 1.05, 1.02], [1.0, 1.0, 1.0]])


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    yield e
    e.close()


def market_at(base, now):
    return W.MarketSpec(list(REALISED[now]), base.sigma, base.corr, base.r,
                        [365 * (t - now) for t in range(now + 1, 6)], now=now,
                        history=[list(REALISED[now - k]) for k in range(1, now + 1)],
                        hist_days=[-365 * k for k in range(1, now + 1)])


def test_one_compile_priced_at_every_valuation_time(eng):
    w = W.worst_of_autocall()
    words, consts = pc.pc_assemble(w.il_text)
    cw, ck = pc.pc_cut_payoff(words, consts)
    cut_text = il_text.to_text(il.cut_payoff(il_text.parse(w.il_text)), [])
    k = pc.pc_load_payoff(eng.ctx, cw, ck, w.tparams, 0, 1)
    eng.contracts.append(k)
    n, seed = 4096 + 3, 0x7E57
    prices = []
    for now in range(5):
        spec = market_at(w.market, now)
        m = eng.model(spec)
        got, sums = eng.paths(m, k, n, seed)
        ref, marg = oracle_paths(cut_text, spec, w.tparams, n, seed)
        compare(got, ref, marg, w.notional, ("now", now))
        assert sums[2] == n
        prices.append(got.mean())
        if now == 0:
            k0 = eng.contract(w.il_text, w.tparams)
            plain, _ = eng.paths(m, k0, n, seed)
            np.testing.assert_array_equal(got, plain)
    # the realised path has a knock-in (0.62 at time 3) and no call until
    # time 4: later valuations see it in the history
    assert len(set(np.round(prices, 6))) == 5
