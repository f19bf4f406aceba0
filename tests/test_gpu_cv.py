"""GPU delta-hedge control variate (pc_price_cv) with caller-supplied hedge
tables.

* per path: the payoff X and the hedge gain M of the kernel against the
  oracle (``oracle.cv``) on identical draws and the same tables;
* the plain half of pc_price_cv is bit-identical to pc_price, and the
  control-variate price agrees with it within the standard errors (E[M] = 0
  for any hedge ratios);
* a European call hedged at 32 dates with tabulated Black-Scholes deltas
  removes most of the variance (the machinery works when the ratios are good).
"""
import math

import numpy as np
import pytest

from gpu_common import Engine, TIE, compare, market, tparam_env, torch
import paper_2108_03076_gb300 as pc
import workloads as W
from oracle import closed_forms as cf, cv, il_text, mc
from oracle.paths import simulate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    yield e
    e.close()


def random_tables(desc, seed):
    """(node records for the device, node ratios [n-1, 2, G^d, d] for the
    oracle): random FP32 ratios, their slopes by the oracle's differences."""
    d, G = desc.d, desc.grid
    rng = np.random.default_rng(seed)
    ratios = (0.3 + 0.4 * rng.standard_normal((desc.n - 1, 2, G ** d, d))).astype(np.float32)
    rec = cv.node_records(ratios.astype(np.float64), G).astype(np.float32)
    assert rec.size == pc.pc_cv_table_size(desc)
    for i in range(3):
        desc.delta0[i] = [0.35, 0.25, 0.15][i]
    return rec.ravel(), ratios.astype(np.float64)


def desc_arrays(desc):
    n, d = desc.n, desc.d
    lo = np.array([[desc.lo[k][i] for i in range(d)] for k in range(max(n - 1, 0))], np.float64)
    h = np.array([[desc.h[k][i] for i in range(d)] for k in range(max(n - 1, 0))], np.float64)
    return lo, h


def test_per_path_payoff_and_hedge_gain_match_oracle(eng):
    w = W.worst_of_autocall()
    m = eng.model(w.market)
    k = eng.contract(w.il_text, w.tparams)
    desc = pc.pc_cv_grid(m, 8, 4.0)
    tab, tables = random_tables(desc, 1)
    dtab = torch.tensor(tab, device="cuda")
    n, seed = 4096 + 13, 0x5EED0101
    xm = torch.empty(3 * n, dtype=torch.float32, device="cuda")
    pc.pc_debug_cv_paths(m, k, desc, dtab.data_ptr(), n, seed, xm.data_ptr())
    torch.cuda.synchronize()
    got = xm.double().cpu().numpy().reshape(n, 3)
    mk = market(w.market)
    x_ref, marg = mc.payoffs(il_text.parse(w.il_text), mk, tparam_env(w.tparams), 0, 1, n, seed, 0, 0,
                             with_margins=True)
    compare(got[:, 0], x_ref, marg, w.notional, "payoff")
    S = np.moveaxis(simulate(mk, seed, 0, np.arange(n)), 1, 2)
    alive, ki = cv.autocall_states(S, [1.0, 1.0, 1.0], 1.0, 0.6)
    lo, h = desc_arrays(desc)
    d, G = desc.d, desc.grid
    delta = cv.table_deltas_taylor(S, ki, tables, lo, h, G, [desc.delta0[i] for i in range(d)])
    disc = [mk.disc(o) for o in range(mk.n + 1)]
    M_ref = cv.hedge_martingale(S, disc, alive, delta)
    worst = S.min(axis=2)[:, 1:mk.n]
    amb = (np.abs(worst - 1.0) < TIE).any(1) | (np.abs(worst - 0.6) < TIE).any(1)
    # a path whose grid coordinate lies within 1e-4 of a half-integer may take
    # the neighbouring node (FP32 against FP64 coordinates)
    u = np.clip((np.log(S[:, 1:mk.n, :]) - lo[None]) / h[None], 0.0, G - 1.0)
    edge = (np.abs(u - np.floor(u) - 0.5) < 1e-4).any((1, 2))
    bad = np.abs(got[:, 1] - M_ref) > 1e-4 * (1.0 + np.abs(M_ref))
    assert not np.any(bad & ~(amb | edge)), np.nonzero(bad & ~(amb | edge))[0][:5]
    assert int((bad & (amb | edge)).sum()) <= max(2, 1e-3 * n)
    assert np.std(M_ref) > 0.05
    # second-order term: gamma from the nearest node's slopes
    gam = cv.table_gammas_taylor(S, ki, tables, lo, h, G)
    tau = [0.0] + [dd / 365.0 for dd in mk.days]
    M2_ref = cv.gamma_martingale(S, disc, alive, gam, np.asarray(mk.corr), mk.sigma, tau)
    bad2 = np.abs(got[:, 2] - M2_ref) > 2e-4 * (1.0 + np.abs(M2_ref))
    assert not np.any(bad2 & ~(amb | edge)), np.nonzero(bad2 & ~(amb | edge))[0][:5]
    assert int((bad2 & (amb | edge)).sum()) <= max(2, 1e-3 * n)
    assert np.std(M2_ref) > 1e-3


@pytest.mark.parametrize("gamma", [0, 1])
def test_plain_half_is_pc_price_and_cv_is_unbiased(eng, gamma):
    w = W.worst_of_autocall()
    m = eng.model(w.market)
    k = eng.contract(w.il_text, w.tparams)
    desc = pc.pc_cv_grid(m, 12, 4.5)
    desc.use_gamma = gamma
    dtab = torch.tensor(random_tables(desc, 2)[0], device="cuda")
    n, seed = 1 << 20, 0x5EED0002
    (pcv, scv), (pp, sp) = pc.pc_price_cv(m, k, desc, dtab.data_ptr(), n, seed)
    price, se = pc.pc_price(m, k, n, seed)
    assert pp == price and sp == se
    assert abs(pcv - pp) <= 4 * (scv + sp), (pcv, pp, scv, sp)
    # betas from a pilot on another seed; beta = 0 gives back the plain estimate
    b1, b2 = pc.pc_cv_beta(m, k, desc, dtab.data_ptr(), 1 << 16, seed + 1)
    assert np.isfinite(b1) and (b2 == 0.0) == (gamma == 0)
    desc.beta, desc.beta2 = 0.0, 0.0
    (p0, s0), _ = pc.pc_price_cv(m, k, desc, dtab.data_ptr(), n, seed)
    assert p0 == pytest.approx(pp, rel=1e-12) and s0 == pytest.approx(sp, rel=1e-9)


def test_black_scholes_hedged_call_removes_most_variance(eng):
    days = [int(round(365 * (j + 1) / 32)) for j in range(32)]
    spec = W.MarketSpec([1.0], [0.2], [[1.0]], 0.03, days)
    m = eng.model(spec)
    k = eng.contract(W.european_text(1.0), [32])
    desc = pc.pc_cv_grid(m, 64, 5.0, ref=(1.0,), call_level=1e30, ki_level=-1.0)
    lo, h = desc_arrays(desc)
    tau = np.array([0.0] + [dd / 365.0 for dd in days])
    ratios = np.zeros((31, 2, 64, 1))
    for kk in range(1, 32):
        y = lo[kk - 1, 0] + h[kk - 1, 0] * np.arange(64)
        dl = np.array([cf.bs_delta_call(math.exp(v), 1.0, 0.03, 0.2, tau[-1] - tau[kk]) for v in y])
        ratios[kk - 1, 0, :, 0] = dl
        ratios[kk - 1, 1, :, 0] = dl
    desc.delta0[0] = cf.bs_delta_call(1.0, 1.0, 0.03, 0.2, tau[-1])
    dtab = torch.tensor(cv.node_records(ratios, 64).ravel().astype(np.float32), device="cuda")
    (pcv, scv), (pp, sp) = pc.pc_price_cv(m, k, desc, dtab.data_ptr(), 1 << 20, 0x5EED0003)
    assert (sp / scv) ** 2 > 8.0, (sp, scv)
    bs = cf.bs_call(1.0, 1.0, 0.03, 0.2, tau[-1])
    assert abs(pcv - bs) < 4 * scv + 1e-4, (pcv, bs, scv)
    # the second-order term from the table's slopes removes more
    desc.use_gamma = 1
    (pg, sg), _ = pc.pc_price_cv(m, k, desc, dtab.data_ptr(), 1 << 20, 0x5EED0003)
    assert sg < scv, (sg, scv)
    assert abs(pg - bs) < 4 * sg + 1e-4, (pg, bs, sg)
