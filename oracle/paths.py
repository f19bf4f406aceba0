"""Path generator: Philox4x32-10, uniforms, Box-Muller, Brownian bridge,
Cholesky correlation and geometric Brownian motion (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper prices with a Monte Carlo engine it does not specify (Sec. 6.2);
the scheme below is the one the GPU engine implements, restated plainly:

* Philox4x32-10: the counter-based generator of Salmon, Moraes, Dror & Shaw,
  "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11), from its published
  definition: 10 rounds, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key
  increments 0x9E3779B9 / 0xBB67AE85, key bumped between rounds.
* normal number m of a path comes from Philox counter (m >> 2, path_lo,
  path_hi, stream), key (seed_lo, seed_hi), output word m & 3.  Bridge node
  j takes the d normals m = d k_j + i (underlying i < d), where k_j is the
  node's rank in the order a date-ordered walk of the bridge computes the
  nodes (``generation_order``): the normals are used in counter order, four
  per Philox block, with none left over.
* uniform u = ((x >> 8) + 0.5) * 2^-24 for a 32-bit output x.
* Box-Muller on the word pairs (0,1) and (2,3): with u_a the even word and
  u_b the odd word, r = sqrt(-2 ln u_a); the even word's normal is
  r cos(2 pi u_b), the odd word's r sin(2 pi u_b).
* Brownian bridge: breadth-first bisection over the date ordinals.  Node 0
  is the last date n, W_n = sqrt(tau_n) z_0; then intervals (l, r) are taken
  from a FIFO starting with (0, n); each with r - l >= 2 gets node
  m = floor((l + r) / 2):
  W_m = w_l W_l + w_r W_r + sd z_j with w_l = (tau_r - tau_m) / (tau_r - tau_l),
  w_r = (tau_m - tau_l) / (tau_r - tau_l),
  sd = sqrt((tau_m - tau_l)(tau_r - tau_m) / (tau_r - tau_l)),
  and pushes (l, m), (m, r).  W_0 = 0 at the valuation date.
* correlation: X = L W with L the Cholesky factor of the correlation matrix.
* GBM: S_i(t_o) = S0_i exp((r - sigma_i^2 / 2) tau_o + sigma_i X_i(t_o)),
  tau_o = day_o / 365 (ACT/365), tau_0 = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF


def _mulhilo(a: int, x: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    p = np.uint64(a) * x.astype(np.uint64)
    return p >> np.uint64(32), p & np.uint64(MASK32)


def philox4x32_10(ctr: Sequence[np.ndarray], key: Tuple[int, int]) -> List[np.ndarray]:
    """Philox4x32-10 of the counter words ``ctr`` (four uint arrays, broadcast
    together) under ``key`` = (k0, k1).  Returns four uint64 arrays holding
    32-bit outputs."""
    x = [np.asarray(c, dtype=np.uint64) & np.uint64(MASK32) for c in ctr]
    x = list(np.broadcast_arrays(*x))
    k0, k1 = int(key[0]) & MASK32, int(key[1]) & MASK32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        hi0, lo0 = _mulhilo(PHILOX_M0, x[0])
        hi1, lo1 = _mulhilo(PHILOX_M1, x[2])
        x = [hi1 ^ x[1] ^ np.uint64(k0), lo1, hi0 ^ x[3] ^ np.uint64(k1), lo0]
    return x


def u24(x: np.ndarray) -> np.ndarray:
    """Uniform in (0, 1) from the top 24 bits of a 32-bit word (exact in FP64)."""
    return ((x.astype(np.uint64) >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24


def box_muller(ua: np.ndarray, ub: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(r cos 2 pi u_b, r sin 2 pi u_b) with r = sqrt(-2 ln u_a)."""
    r = np.sqrt(-2.0 * np.log(ua))
    th = 2.0 * math.pi * ub
    return r * np.cos(th), r * np.sin(th)


def split_seed(seed: int) -> Tuple[int, int]:
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & MASK32, seed >> 32


def normals(seed: int, stream: int, paths: np.ndarray, count: int) -> np.ndarray:
    """Normals number 0..count-1 of each path in ``paths`` (uint64 global path
    indices).  Returns float64 [len(paths), count]."""
    paths = np.asarray(paths, dtype=np.uint64)
    p_lo = paths & np.uint64(MASK32)
    p_hi = paths >> np.uint64(32)
    key = split_seed(seed)
    nblk = (count + 3) // 4
    out = np.empty((len(paths), 4 * nblk), dtype=np.float64)
    for b in range(nblk):
        x = philox4x32_10([np.uint64(b), p_lo, p_hi, np.uint64(stream & MASK32)], key)
        z0, z1 = box_muller(u24(x[0]), u24(x[1]))
        z2, z3 = box_muller(u24(x[2]), u24(x[3]))
        out[:, 4 * b + 0] = z0
        out[:, 4 * b + 1] = z1
        out[:, 4 * b + 2] = z2
        out[:, 4 * b + 3] = z3
    return out[:, :count]


# ---------------------------------------------------------------------------
# Brownian bridge (array form)
# ---------------------------------------------------------------------------


@dataclass
class BridgeNode:
    m: int          # date ordinal produced
    l: int          # left endpoint ordinal (0 for the root)
    r: int          # right endpoint ordinal (-1 for the root)
    wl: float
    wr: float
    sd: float


def bridge_schedule(tau: Sequence[float]) -> List[BridgeNode]:
    """Breadth-first bisection schedule over ordinals 0..n with year
    fractions ``tau`` (tau[0] = 0).  Node j of the list uses normal block j."""
    n = len(tau) - 1
    if n < 1:
        return []
    nodes = [BridgeNode(n, 0, -1, 0.0, 0.0, math.sqrt(tau[n] - tau[0]))]
    queue = [(0, n)]
    head = 0
    while head < len(queue):
        l, r = queue[head]
        head += 1
        if r - l < 2:
            continue
        m = (l + r) // 2
        span = tau[r] - tau[l]
        nodes.append(BridgeNode(m, l, r, (tau[r] - tau[m]) / span,
                                (tau[m] - tau[l]) / span,
                                math.sqrt((tau[m] - tau[l]) * (tau[r] - tau[m]) / span)))
        queue.append((l, m))
        queue.append((m, r))
    return nodes


def generation_order(nodes: List[BridgeNode]) -> np.ndarray:
    """Rank of each node in the order a walk that produces the dates in
    increasing order computes them.  To produce date t from the last
    produced date t - 1, the walk needs W at the nearest later date already
    computed, and bisects towards t: it computes every node whose bisection
    interval starts at t - 1, the widest interval (largest midpoint) first.
    The root (date n) is computed first, with the nodes of intervals
    starting at 0.  So the rank orders nodes by (left end, -date)."""
    keys = [(nd.l, -nd.m) for nd in nodes]
    order = sorted(range(len(nodes)), key=lambda j: keys[j])
    rank = np.empty(len(nodes), dtype=np.int64)
    rank[np.asarray(order, dtype=np.int64)] = np.arange(len(nodes))
    return rank


def node_normals(nodes: List[BridgeNode], d: int, seed: int, stream: int,
                 paths: np.ndarray) -> np.ndarray:
    """z[p, j, i]: normal of underlying i at bridge node j, i.e. normal
    number d k_j + i of the path (k = ``generation_order``)."""
    n = len(nodes)
    z = normals(seed, stream, paths, n * d).reshape(len(paths), n, d)     # [p, k, i]
    return z[:, generation_order(nodes), :]


def bridge_apply(nodes: List[BridgeNode], z: np.ndarray, n: int) -> np.ndarray:
    """W[..., o] for o = 0..n from normals z[..., j] (one per node)."""
    W = np.zeros(z.shape[:-1] + (n + 1,), dtype=np.float64)
    for j, nd in enumerate(nodes):
        if nd.r < 0:
            W[..., nd.m] = nd.sd * z[..., j]
        else:
            W[..., nd.m] = nd.wl * W[..., nd.l] + nd.wr * W[..., nd.r] + nd.sd * z[..., j]
    return W


# ---------------------------------------------------------------------------
# Market model
# ---------------------------------------------------------------------------


@dataclass
class Market:
    """Correlated Black-Scholes market on a date grid.

    ``days[k-1]`` is the calendar day (relative to the valuation date) of
    ordinal k = 1..n; ordinal 0 is the valuation date.  ``now`` is the IL time
    of the valuation date: IL time t is ordinal t - now.  Ordinals -1, -2, ...
    are history: ``history[k-1][l]`` is label l at ordinal -k and
    ``hist_days[k-1]`` its (negative) day.
    """
    S0: Sequence[float]
    sigma: Sequence[float]
    corr: Sequence[Sequence[float]]
    r: float
    days: Sequence[int]
    now: int = 0
    history: Sequence[Sequence[float]] = field(default_factory=list)
    hist_days: Sequence[int] = field(default_factory=list)

    @property
    def d(self) -> int:
        return len(self.S0)

    @property
    def n(self) -> int:
        return len(self.days)

    def tau(self) -> np.ndarray:
        """Year fractions of ordinals 0..n (ACT/365)."""
        return np.concatenate([[0.0], np.asarray(self.days, dtype=np.float64) / 365.0])

    def cholesky(self) -> np.ndarray:
        return np.linalg.cholesky(np.asarray(self.corr, dtype=np.float64))

    def disc(self, t: int) -> float:
        """d(t) = exp(-r tau) at IL time t (ordinal t - now)."""
        o = t - self.now
        if o >= 0:
            if o > self.n:
                raise IndexError(f"payoff time {t} beyond the date grid")
            return math.exp(-self.r * self.tau()[o])
        k = -o
        if k > len(self.hist_days):
            raise IndexError(f"payoff time {t} before the history")
        return math.exp(-self.r * self.hist_days[k - 1] / 365.0)


def simulate_sx(mk: Market, seed: int, stream: int, paths: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(S[p, i, o], X[p, i, o]) for the paths ``paths`` (global indices),
    o = 0..n: the prices and the correlated Brownian values X = L W."""
    n, d = mk.n, mk.d
    paths = np.asarray(paths, dtype=np.uint64)
    tau = mk.tau()
    nodes = bridge_schedule(tau)
    z = node_normals(nodes, d, seed, stream, paths)                     # [p, j, i]
    W = bridge_apply(nodes, np.moveaxis(z, 2, 1), n)                     # [p, i, o]
    L = mk.cholesky()
    X = np.einsum("ik,pko->pio", L, W)
    sig = np.asarray(mk.sigma, dtype=np.float64)[None, :, None]
    S0 = np.asarray(mk.S0, dtype=np.float64)[None, :, None]
    return S0 * np.exp((mk.r - 0.5 * sig ** 2) * tau[None, None, :] + sig * X), X


def simulate(mk: Market, seed: int, stream: int, paths: np.ndarray) -> np.ndarray:
    """S[p, i, o] for the paths ``paths`` (global indices), o = 0..n."""
    return simulate_sx(mk, seed, stream, paths)[0]


def simulate_from_normals(mk: Market, z: np.ndarray) -> np.ndarray:
    """Same map as ``simulate`` but from given normals z[p, j, i]."""
    n = mk.n
    tau = mk.tau()
    W = bridge_apply(bridge_schedule(tau), np.moveaxis(z, 2, 1), n)
    X = np.einsum("ik,pko->pio", mk.cholesky(), W)
    sig = np.asarray(mk.sigma, dtype=np.float64)[None, :, None]
    S0 = np.asarray(mk.S0, dtype=np.float64)[None, :, None]
    return S0 * np.exp((mk.r - 0.5 * sig ** 2) * tau[None, None, :] + sig * X)
