"""Learned control variate for the worst-of autocallable template.

A network (16 inputs -> 256 -> 256 -> 256 -> 5 outputs: value and hedge
ratios of the remaining contract) is trained on prices and sensitivities
that the engine itself computes, then tabulated over the simulated states
and used as the hedge of the delta-hedge control variate of
``pc_price_cv``: Y = X - sum_k Delta(k) . (D_{k+1} S_{k+1} - D_k S_k) has
the price as its mean for any hedge ratios, so the network only decides
how much variance is removed; plain Monte Carlo (the X half of the same
launch) is the unbiased check on the result.

Training data: random template parameters and states (observation date k,
spots S relative to the reference levels, knock-in flag).  Each sample's
remaining contract (the autocall from date k on, with its coupons and the
knock-in already seen) is priced by the engine's portfolio plans: one plan
at the state and six at spots bumped by +-h per underlying on the same
Philox streams (common random numbers), giving value and central-difference
hedge ratios.  Everything numeric runs in the library's kernels; this
module builds program texts and feature rows and moves arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np

from . import (pc_assemble, pc_batch_create, pc_batch_destroy, pc_batch_launch, pc_batch_results,
               pc_contract_destroy, pc_cv_beta, pc_cv_grid, pc_cv_labels, pc_cv_table_size, pc_cv_tables,
               pc_cv_tables_async, pc_load_payoff, pc_mlp_create, pc_mlp_destroy, pc_mlp_forward, pc_mlp_train, pc_model_create,
               pc_model_destroy, pc_price_cv)

WIDTHS = (16, 256, 256, 256, 5)
N_DATES = 5
D = 3


def _fmt(x: float) -> str:
    r = repr(float(x))
    return r if any(c in r for c in ".eE") else r + ".0"


def autocall_state_text(n_rem: int, k_elapsed: int, coupon: float, call_level: float,
                        ki_level: float, ki_flag: bool, d: int = D) -> str:
    """Program of the worst-of autocallable from observation date k_elapsed
    on (n_rem dates left, at ordinals 1..n_rem of a model starting at that
    date; reference levels 1): at date j < n_rem pay 1 + coupon (k + j) and
    stop if worst >= call_level; at the last date pay 1 + coupon n if
    worst >= call_level, else worst if knocked in (flag or some remaining
    worst <= ki_level), else 1."""
    def W(j: int) -> str:
        out = f"(model 0 {j})"
        for i in range(1, d):
            out = f"(min {out} (model {i} {j}))"
        return out

    def pay(j: int) -> str:
        return f"(payoff {j} 0 1)"

    n, kk = n_rem, k_elapsed
    if ki_flag:
        maturity_else = f"(mult {W(n)} {pay(n)})"
    else:
        kis = [f"(le {W(n - j)} {_fmt(ki_level)})" for j in range(n)]
        ki = kis[-1]
        for x in reversed(kis[:-1]):
            ki = f"(or {x} {ki})"
        maturity_else = f"(mult (if {ki} {W(n)} 1.0) {pay(n)})"
    body = (f"(loopif (le {_fmt(call_level)} {W(n)}) "
            f"(mult {_fmt(1.0 + coupon * (kk + n))} {pay(n)}) {maturity_else} 0)")
    for j in range(n - 1, 0, -1):
        body = (f"(loopif (le {_fmt(call_level)} {W(j)}) "
                f"(mult {_fmt(1.0 + coupon * (kk + j))} {pay(j)}) {body} 0)")
    return body


def features(lnS: np.ndarray, ki: np.ndarray, k: np.ndarray, n: int, sigma: np.ndarray, rho: np.ndarray,
             r: np.ndarray, dt_next: np.ndarray, coupon: np.ndarray, call_level: np.ndarray,
             ki_level: np.ndarray) -> np.ndarray:
    """Network input rows [N, 16] (the layout pc_cv_tables builds on the
    device): ln(S_i / ref_i), sigma_i, rho, r, time to the next date,
    remaining dates / 5, elapsed dates / 5, knock-in, coupon, call level,
    knock-in level, 1.  Arguments are per-row arrays (or broadcastable)."""
    N = lnS.shape[0]
    F = np.zeros((N, 16), np.float64)
    F[:, :D] = lnS
    F[:, 3:3 + D] = sigma
    F[:, 6] = rho
    F[:, 7] = r
    F[:, 8] = dt_next
    F[:, 9] = (n - np.asarray(k)) / 5.0
    F[:, 10] = np.asarray(k) / 5.0
    F[:, 11] = np.asarray(ki, np.float64)
    F[:, 12] = coupon
    F[:, 13] = call_level
    F[:, 14] = ki_level
    F[:, 15] = 1.0
    return F


@dataclass
class TrainingSet:
    x: np.ndarray        # [N, 16] features
    y: np.ndarray        # [N, 5] value, hedge ratios (3), 0
    paths: int           # engine paths per sample


def sample_states(n: int, rng: np.random.Generator):
    """Template parameters and reachable states of the remaining contract."""
    sig = rng.uniform(0.15, 0.35, (n, D))
    rho = rng.uniform(0.3, 0.7, n)
    r = rng.uniform(0.01, 0.05, n)
    coupon = rng.uniform(0.03, 0.07, n)
    call = rng.uniform(0.95, 1.05, n)
    kil = rng.uniform(0.5, 0.7, n)
    k = rng.integers(0, N_DATES, n)
    lnS = np.zeros((n, D))
    ki = np.zeros(n, bool)
    for c in range(n):
        if k[c] == 0:
            lnS[c] = rng.normal(0.0, 0.08, D)
            continue
        for _ in range(100):
            t = float(k[c])
            lnS[c] = (r[c] - 0.5 * sig[c] ** 2) * t + 1.3 * sig[c] * math.sqrt(t) * rng.normal(size=D)
            if np.exp(lnS[c]).min() < call[c]:
                break
        worst = np.exp(lnS[c]).min()
        ki[c] = worst <= kil[c] or rng.uniform() < 0.25
    return dict(sig=sig, rho=rho, r=r, coupon=coupon, call=call, kil=kil, k=k, lnS=lnS, ki=ki)


def engine_training_set(ctx: int, n_samples: int, paths: int, seed: int, bump: float = 0.02,
                        rng_seed: int = 0x1EA4) -> TrainingSet:
    """Values and CRN central-difference hedge ratios of sampled states,
    priced by the engine (seven portfolio plans over the same contracts)."""
    rng = np.random.Generator(np.random.MT19937(rng_seed))
    st = sample_states(n_samples, rng)
    contracts, models = [], [[] for _ in range(2 * D + 1)]
    try:
        for c in range(n_samples):
            n_rem = N_DATES - int(st["k"][c])
            text = autocall_state_text(n_rem, int(st["k"][c]), st["coupon"][c], st["call"][c],
                                       st["kil"][c], bool(st["ki"][c]))
            w, kc = pc_assemble(text)
            contracts.append(pc_load_payoff(ctx, w, kc, []))
            corr = [[1.0 if i == j else float(st["rho"][c]) for j in range(D)] for i in range(D)]
            days = [365 * (j + 1) for j in range(n_rem)]
            S = np.exp(st["lnS"][c])
            for b in range(2 * D + 1):
                Sb = S.copy()
                if b:
                    i, sgn = (b - 1) // 2, (1.0 if (b - 1) % 2 == 0 else -1.0)
                    Sb[i] *= 1.0 + sgn * bump
                models[b].append(pc_model_create(ctx, Sb, st["sig"][c], corr, float(st["r"][c]), days))
        prices = []
        for b in range(2 * D + 1):
            plan = pc_batch_create(models[b], contracts, [paths] * n_samples, seed)
            try:
                pc_batch_launch(plan)
                prices.append(pc_batch_results(plan, n_samples)[0])
            finally:
                pc_batch_destroy(plan)
    finally:
        for ms in models:
            for m in ms:
                pc_model_destroy(m)
        for kc in contracts:
            pc_contract_destroy(kc)
    y = pc_cv_labels(np.stack(prices), np.exp(st["lnS"]), bump, 5)
    x = features(st["lnS"], st["ki"], st["k"], N_DATES, st["sig"], st["rho"], st["r"],
                 np.ones(n_samples), st["coupon"], st["call"], st["kil"])
    return TrainingSet(x.astype(np.float32), y.astype(np.float32), paths)


class LearnedCV:
    """The trained network and its use as the hedge of pc_price_cv."""

    def __init__(self, ctx: int, seed: int = 7, max_batch: int = 16384):
        self.ctx = ctx
        self.net = pc_mlp_create(ctx, WIDTHS, max_batch, seed)
        self.betas = (1.0, 1.0)     # (beta, beta2) for the hedge terms; see calibrate()

    def close(self):
        if self.net:
            pc_mlp_destroy(self.net)
            self.net = 0

    def train(self, data: TrainingSet, steps: int, batch: int = 1024, lr: float = 1e-3,
              delta_weight: float = 0.1, seed: int = 11) -> Tuple[float, float]:
        """Adam on the engine-generated set; returns (first, last) minibatch loss."""
        import torch
        dx = torch.tensor(data.x, device="cuda")
        dy = torch.tensor(data.y, device="cuda")
        w = np.array([1.0, delta_weight, delta_weight, delta_weight, 0.0], np.float32)
        first = pc_mlp_train(self.net, dx.data_ptr(), dy.data_ptr(), len(data.x), w, batch, 1, lr, seed)
        last = first
        done = 1
        while done < steps:
            chunk = min(1000, steps - done)
            rate = lr * (0.1 if done > 0.75 * steps else 1.0)
            last = pc_mlp_train(self.net, dx.data_ptr(), dy.data_ptr(), len(data.x), w, batch, chunk,
                                rate, seed)
            done += chunk
        return first, last

    def predict(self, x: np.ndarray) -> np.ndarray:
        import torch
        dx = torch.tensor(np.asarray(x, np.float32), device="cuda")
        dy = torch.empty((len(x), 5), dtype=torch.float32, device="cuda")
        pc_mlp_forward(self.net, dx.data_ptr(), len(x), dy.data_ptr())
        torch.cuda.synchronize()
        return dy.cpu().numpy()

    def tables(self, model: int, grid: int = 12, width_sd: float = 4.5, call_level: float = 1.0,
               ki_level: float = 0.6, coupon: float = 0.05, gamma: bool = True, out=None,
               asynchronous: bool = False):
        """(description, device tables) for a model of the template, with the
        calibrated betas (and the second-order term when ``gamma``).  ``out``:
        a float32 CUDA tensor to fill (large enough), else a new one; rebuilding
        into the same buffer replays the build's captured graph.
        ``asynchronous``: enqueue the build without waiting; delta0 stays on
        the device after the tables (pc_cv_tables_async)."""
        import torch
        desc = pc_cv_grid(model, grid, width_sd, (1.0, 1.0, 1.0), call_level, ki_level, coupon)
        n = pc_cv_table_size(desc)
        dt = out if out is not None and out.numel() >= n + 4 else torch.empty(n + 4, dtype=torch.float32,
                                                                             device="cuda")
        (pc_cv_tables_async if asynchronous else pc_cv_tables)(self.net, model, desc, dt.data_ptr(), n + 4)
        desc.use_gamma = 1 if gamma else 0
        desc.beta, desc.beta2 = self.betas if gamma else (self.betas_first_order, 0.0)
        return desc, dt

    betas_first_order = 1.0

    def calibrate(self, model: int, contract: int, n_paths: int = 1 << 18, seed: int = 0xCA11B):
        """Fix the betas once for the template: the variance-minimising
        values on a pilot run (its own seed, so later prices use fixed
        betas and stay unbiased)."""
        desc, dt = self.tables(model, gamma=True)
        self.betas = pc_cv_beta(model, contract, desc, dt.data_ptr(), n_paths, seed)
        desc, dt = self.tables(model, gamma=False)
        self.betas_first_order = pc_cv_beta(model, contract, desc, dt.data_ptr(), n_paths, seed)[0]
        return self.betas

    @staticmethod
    def price(model: int, contract: int, desc, d_tables, n_paths: int, seed: int):
        """((price, se) with the control variate, (price, se) plain)."""
        return pc_price_cv(model, contract, desc, d_tables.data_ptr(), n_paths, seed)
