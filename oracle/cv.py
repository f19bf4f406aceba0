"""Delta-hedge control variate for the worst-of autocallable template (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

An extension of the paper's Monte Carlo valuation (Sec. 3 averages the
per-path payoff of Fig. 3), not a passage of the paper.  For a contract on
d underlyings observed at dates t_1 < ... < t_n, with discount factors
D_k = exp(-r tau_k) (D_0 = 1) and any hedge ratios Delta_i(k) that depend
only on the path up to t_k,

    M = sum_{k=0}^{n-1} alive_k sum_i Delta_i(k) (D_{k+1} S_i(t_{k+1}) - D_k S_i(t_k))

is a sum of martingale increments under the pricing measure (the discounted
underlyings D S_i are martingales), so E[M] = 0 and Y = X - M is an unbiased
estimator of the price E[X] whatever the Delta's are; the closer Delta is to
the sensitivity of the contract's value at t_k, the smaller Var(Y).

Worst-of autocallable states (the template of ``contracts.autocall_cl``):
worst_k = min_i S_i(t_k) / ref_i; the contract is alive over [t_k, t_{k+1}]
if it was not called at any date j <= k (j < n) by worst_j >= call_level;
the knock-in flag at t_k is "some worst_j <= ki_level, 1 <= j <= k".

Hedge ratios come from a table over y = ln S at each date k = 1..n-1 and
knock-in state (k = 0 has the single value ``delta0``), read by
multilinear interpolation: per axis u = clamp((y - lo) / h, 0, G - 1),
a = min(floor(u), G - 2), f = u - a; the value is the sum over the 2^d
cell corners of prod_axis (f or 1 - f) times the corner entry.  Table
layout [k - 1][ki][node][i] with node = ((a_0 G + a_1) G + a_2) (asset 0
slowest), d values per node.

Second-order (gamma) term: with X_i = D_{k+1} S_i(t_{k+1}) - D_k S_i(t_k)
and any adapted symmetric Gamma(k),

    M2 = sum_{k>=1} alive_k 1/2 sum_ij Gamma_ij(k) (X_i X_j - E_k[X_i X_j]),
    E_k[X_i X_j] = D_k^2 S_i(t_k) S_j(t_k) (exp(rho_ij sigma_i sigma_j dt_k) - 1)

(the discounted returns D_{k+1} S_{k+1} / (D_k S_k) are lognormal with mean
1 and E[R_i R_j] = exp(rho_ij sigma_i sigma_j dt)), so E[M2] = 0 as well.
Gamma comes from the slopes of the multilinear hedge-ratio table: along
axis j the interpolant's derivative s_ij = d Delta_i / d u_j (u_j = (ln S_j
- lo_j) / h_j), Gamma_ij = (s_ij / (h_j S_j) + s_ji / (h_i S_i)) / 2.

Network features of a state (the 16 inputs of the learned model):
ln(S_i / ref_i) for i < 3 (0 beyond d), sigma_i for i < 3, rho, r, the time
to the next date (years), remaining dates / 5, elapsed dates / 5, knock-in
flag, coupon, call level, knock-in level, 1.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np

N_FEATURES = 16
N_OUTPUTS = 5


def autocall_states(S: np.ndarray, ref: Sequence[float], call_level: float,
                    ki_level: float) -> Tuple[np.ndarray, np.ndarray]:
    """S: [N, n+1, d] path values at t_0..t_n.  Returns alive [N, n] and
    ki [N, n] (states at t_0..t_{n-1})."""
    N, n1, d = S.shape
    n = n1 - 1
    worst = (S / np.asarray(ref)[None, None, :]).min(axis=2)
    alive = np.zeros((N, n), bool)
    ki = np.zeros((N, n), bool)
    a = np.ones(N, bool)
    kf = np.zeros(N, bool)
    for k in range(n):
        if k >= 1:
            kf = kf | (worst[:, k] <= ki_level)
            a = a & ~(worst[:, k] >= call_level)
        alive[:, k] = a
        ki[:, k] = kf
    return alive, ki


def hedge_martingale(S: np.ndarray, disc: Sequence[float], alive: np.ndarray,
                     delta: np.ndarray) -> np.ndarray:
    """M per path; delta [N, n, d] hedge ratios at t_0..t_{n-1}."""
    D = np.asarray(disc, dtype=np.float64)
    n = alive.shape[1]
    M = np.zeros(S.shape[0])
    for k in range(n):
        inc = D[k + 1] * S[:, k + 1, :] - D[k] * S[:, k, :]
        M += np.where(alive[:, k], (delta[:, k, :] * inc).sum(axis=1), 0.0)
    return M


def table_lookup(table: np.ndarray, lo: np.ndarray, h: np.ndarray, G: int,
                 y: np.ndarray) -> np.ndarray:
    """Multilinear interpolation; table [G^d, d], lo/h [d], y [N, d] -> [N, d]."""
    N, d = y.shape
    u = np.clip((y - lo[None, :]) / h[None, :], 0.0, G - 1.0)
    a = np.minimum(np.floor(u).astype(np.int64), G - 2)
    f = u - a
    out = np.zeros((N, d))
    for corner in range(1 << d):
        wgt = np.ones(N)
        node = np.zeros(N, np.int64)
        for ax in range(d):
            bit = (corner >> (d - 1 - ax)) & 1
            wgt = wgt * (f[:, ax] if bit else 1.0 - f[:, ax])
            node = node * G + a[:, ax] + bit
        out += wgt[:, None] * table[node]
    return out


def table_deltas(S: np.ndarray, ki: np.ndarray, tables: np.ndarray, lo: np.ndarray,
                 h: np.ndarray, G: int, delta0: Sequence[float]) -> np.ndarray:
    """Hedge ratios [N, n, d] for every path and date from the tables
    [n-1, 2, G^d, d] (lo, h: [n-1, d]) and delta0 at t_0."""
    N, n1, d = S.shape
    n = n1 - 1
    out = np.zeros((N, n, d))
    out[:, 0, :] = np.asarray(delta0)[None, :]
    for k in range(1, n):
        y = np.log(S[:, k, :])
        for s in (0, 1):
            sel = ki[:, k] == bool(s)
            if sel.any():
                out[sel, k, :] = table_lookup(tables[k - 1, s], lo[k - 1], h[k - 1], G, y[sel])
    return out


def autocall_features(lnS: np.ndarray, ki: np.ndarray, k: int, n: int, sigma: Sequence[float],
                      rho: float, r: float, dt_next: float, coupon: float, call_level: float,
                      ki_level: float) -> np.ndarray:
    """Feature rows [N, 16] of states at date index k (ln S relative to ref)."""
    N, d = lnS.shape
    F = np.zeros((N, N_FEATURES))
    F[:, :d] = lnS
    F[:, 3:3 + d] = np.asarray(sigma)[None, :d]
    F[:, 6] = rho
    F[:, 7] = r
    F[:, 8] = dt_next
    F[:, 9] = (n - k) / 5.0
    F[:, 10] = k / 5.0
    F[:, 11] = ki.astype(np.float64)
    F[:, 12] = coupon
    F[:, 13] = call_level
    F[:, 14] = ki_level
    F[:, 15] = 1.0
    return F


def table_slopes(table: np.ndarray, lo: np.ndarray, h: np.ndarray, G: int,
                 y: np.ndarray) -> np.ndarray:
    """d (interpolated Delta_i) / d u_j on the cell of each point: [N, d, d]
    (same clamping and cell choice as ``table_lookup``)."""
    N, d = y.shape
    u = np.clip((y - lo[None, :]) / h[None, :], 0.0, G - 1.0)
    a = np.minimum(np.floor(u).astype(np.int64), G - 2)
    f = u - a
    out = np.zeros((N, d, d))
    for corner in range(1 << d):
        node = np.zeros(N, np.int64)
        bits = []
        for ax in range(d):
            bit = (corner >> (d - 1 - ax)) & 1
            bits.append(bit)
            node = node * G + a[:, ax] + bit
        for j in range(d):
            wgt = np.ones(N)
            for ax in range(d):
                if ax == j:
                    wgt = wgt * (1.0 if bits[ax] else -1.0)
                else:
                    wgt = wgt * (f[:, ax] if bits[ax] else 1.0 - f[:, ax])
            out[:, :, j] += wgt[:, None] * table[node]
    return out


def gamma_martingale(S: np.ndarray, disc: Sequence[float], alive: np.ndarray, gamma: np.ndarray,
                     corr: np.ndarray, sigma: Sequence[float], tau: Sequence[float]) -> np.ndarray:
    """M2 per path; gamma [N, n, d, d] symmetric (entries for k = 0 unused)."""
    D = np.asarray(disc, dtype=np.float64)
    sig = np.asarray(sigma, dtype=np.float64)
    n = alive.shape[1]
    M2 = np.zeros(S.shape[0])
    for k in range(1, n):
        dt = tau[k + 1] - tau[k]
        c = np.exp(np.asarray(corr) * np.outer(sig, sig) * dt) - 1.0
        X = D[k + 1] * S[:, k + 1, :] - D[k] * S[:, k, :]
        q = np.einsum("pi,pij,pj->p", X, gamma[:, k], X)
        e = D[k] ** 2 * np.einsum("pi,pij,pj,ij->p", S[:, k, :], gamma[:, k], S[:, k, :], c)
        M2 += np.where(alive[:, k], 0.5 * (q - e), 0.0)
    return M2


def table_gammas(S: np.ndarray, ki: np.ndarray, tables: np.ndarray, lo: np.ndarray, h: np.ndarray,
                 G: int) -> np.ndarray:
    """Gamma [N, n, d, d] from the table slopes (zero at t_0)."""
    N, n1, d = S.shape
    n = n1 - 1
    out = np.zeros((N, n, d, d))
    for k in range(1, n):
        y = np.log(S[:, k, :])
        for s in (0, 1):
            sel = ki[:, k] == bool(s)
            if not sel.any():
                continue
            sl = table_slopes(tables[k - 1, s], lo[k - 1], h[k - 1], G, y[sel])
            g = sl / (h[k - 1][None, None, :] * S[sel, k, :][:, None, :])
            out[sel, k] = 0.5 * (g + np.swapaxes(g, 1, 2))
    return out


# --- nearest-node Taylor tables -------------------------------------------
# The hedge tables the engine prices with: each node keeps its hedge ratios
# and their slopes along the grid axes (central differences of the node
# values, one-sided on the grid's faces), and a point takes the nearest
# node's ratios plus the first-order step to it, Delta_i(u) = Delta_i(a) +
# sum_j s_ij(a) (u_j - a_j) with a = floor(u + 1/2), u the grid coordinate
# (ln S - lo) / h clamped to [0, G - 1].  Its gamma is the node's slopes
# divided by h_j S_j, symmetrised.  Any such hedge is adapted, so the
# martingales above keep mean zero.


def node_slopes(table: np.ndarray, G: int) -> np.ndarray:
    """Slopes [G^d, d, d] (s[node, i, j] = d Delta_i / d u_j) of a table
    [G^d, d] by central differences along each axis, one-sided at the ends."""
    nodes, d = table.shape
    T = table.reshape((G,) * d + (d,))
    out = np.zeros((G,) * d + (d, d))
    for j in range(d):
        fwd = np.take(T, np.minimum(np.arange(G) + 1, G - 1), axis=j)
        bwd = np.take(T, np.maximum(np.arange(G) - 1, 0), axis=j)
        span = np.where((np.arange(G) == 0) | (np.arange(G) == G - 1), 1.0, 2.0)
        shape = [1] * d + [1]
        shape[j] = G
        out[..., :, j] = (fwd - bwd) / span.reshape(shape)
    return out.reshape(nodes, d, d)


def taylor_lookup(table: np.ndarray, slopes: np.ndarray, lo: np.ndarray, h: np.ndarray, G: int,
                  y: np.ndarray):
    """(Delta [N, d], slopes [N, d, d]) at points y [N, d] from the nearest node."""
    N, d = y.shape
    u = np.clip((y - lo[None, :]) / h[None, :], 0.0, G - 1.0)
    a = np.floor(u + 0.5).astype(np.int64)
    node = np.zeros(N, np.int64)
    for ax in range(d):
        node = node * G + a[:, ax]
    s = slopes[node]
    return table[node] + np.einsum("pij,pj->pi", s, u - a), s


def table_deltas_taylor(S: np.ndarray, ki: np.ndarray, tables: np.ndarray, lo: np.ndarray,
                        h: np.ndarray, G: int, delta0: Sequence[float]) -> np.ndarray:
    """``table_deltas`` with nearest-node Taylor tables (node values tables
    [n-1, 2, G^d, d], slopes by ``node_slopes``)."""
    N, n1, d = S.shape
    n = n1 - 1
    out = np.zeros((N, n, d))
    out[:, 0, :] = np.asarray(delta0)[None, :]
    for k in range(1, n):
        y = np.log(S[:, k, :])
        for s in (0, 1):
            sel = ki[:, k] == bool(s)
            if sel.any():
                sl = node_slopes(tables[k - 1, s], G)
                out[sel, k, :] = taylor_lookup(tables[k - 1, s], sl, lo[k - 1], h[k - 1], G, y[sel])[0]
    return out


def table_gammas_taylor(S: np.ndarray, ki: np.ndarray, tables: np.ndarray, lo: np.ndarray,
                        h: np.ndarray, G: int) -> np.ndarray:
    """``table_gammas`` with nearest-node Taylor tables: the node's slopes."""
    N, n1, d = S.shape
    n = n1 - 1
    out = np.zeros((N, n, d, d))
    for k in range(1, n):
        y = np.log(S[:, k, :])
        for s in (0, 1):
            sel = ki[:, k] == bool(s)
            if not sel.any():
                continue
            sl = node_slopes(tables[k - 1, s], G)
            g = taylor_lookup(tables[k - 1, s], sl, lo[k - 1], h[k - 1], G, y[sel])[1]
            g = g / (h[k - 1][None, None, :] * S[sel, k, :][:, None, :])
            out[sel, k] = 0.5 * (g + np.swapaxes(g, 1, 2))
    return out


def node_records(tables: np.ndarray, G: int) -> np.ndarray:
    """The engine's table layout from node values [n-1, 2, G^d, d]: per node
    12 floats, Delta_0..2 then s_ij at 3 + 3 i + j (zero beyond d)."""
    m, two, nodes, d = tables.shape
    rec = np.zeros((m, two, nodes, 12))
    for a in range(m):
        for b in range(two):
            sl = node_slopes(tables[a, b], G)
            rec[a, b, :, :d] = tables[a, b]
            for i in range(d):
                for j in range(d):
                    rec[a, b, :, 3 + 3 * i + j] = sl[:, i, j]
    return rec
