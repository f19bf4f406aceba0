"""Pins of the oracle's learned-control-variate parts.

MLP: a one-unit network against its formula written out, softplus special
values, backpropagated gradients against central finite differences of the
FP64 loss (all parameters of a small network), the input gradient likewise,
and Adam's first step (a step of lr against the gradient's sign).

Control variate: the autocall states on hand-made paths, the hedge
martingale has mean zero for an arbitrary adapted hedge, a European call
hedged daily with its Black-Scholes delta replicates the payoff (variance
nearly removed), and multilinear interpolation reproduces multilinear
functions exactly and clamps outside the grid.  Second-order term: mean
zero for an arbitrary adapted gamma, a quarterly delta+gamma hedge of a
call (closed-form gamma) beats delta alone, and the table slopes are the
interpolant's derivatives (central differences).
"""
import math

import numpy as np
import pytest

from oracle import closed_forms as cf, cv, mlp
from oracle.paths import Market, simulate


def test_softplus_and_sigmoid_values():
    assert mlp.softplus(np.array(0.0)) == pytest.approx(math.log(2.0), rel=1e-15)
    assert mlp.sigmoid(np.array(0.0)) == 0.5
    z = np.linspace(-30, 30, 61)
    h = 1e-5
    fd = (mlp.softplus(z + h) - mlp.softplus(z - h)) / (2 * h)
    np.testing.assert_allclose(fd, mlp.sigmoid(z), atol=1e-9)
    assert mlp.softplus(np.array(800.0)) == pytest.approx(800.0)


def test_one_unit_network_by_hand():
    params = [(np.array([[1.5, -2.0]]), np.array([0.25])), (np.array([[3.0]]), np.array([-1.0]))]
    x = np.array([[0.2, 0.7], [-1.0, 0.0]])
    y, _ = mlp.forward(params, x)
    want = [3.0 * math.log1p(math.exp(1.5 * a - 2.0 * b + 0.25)) - 1.0 for a, b in x]
    np.testing.assert_allclose(y[:, 0], want, rtol=1e-14)


@pytest.fixture
def small():
    rng = np.random.default_rng(7)
    params = mlp.init([4, 7, 6, 3], rng)
    x = rng.normal(size=(5, 4))
    t = rng.normal(size=(5, 3))
    w = np.array([1.0, 0.5, 2.0])
    return params, x, t, w


def test_backprop_matches_finite_differences(small):
    params, x, t, w = small
    L, grads = mlp.backward(params, x, t, w)
    assert L == pytest.approx(mlp.loss(params, x, t, w), rel=1e-15)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for k, P in enumerate((W, b)):
            fd = np.zeros_like(P)
            for idx in np.ndindex(P.shape):
                old = P[idx]
                P[idx] = old + h
                up = mlp.loss(params, x, t, w)
                P[idx] = old - h
                dn = mlp.loss(params, x, t, w)
                P[idx] = old
                fd[idx] = (up - dn) / (2 * h)
            np.testing.assert_allclose(grads[l][k], fd, rtol=1e-6, atol=1e-9)


def test_input_gradient_matches_finite_differences(small):
    params, x, _, _ = small
    for j in range(3):
        g = mlp.input_gradient(params, x, j)
        h = 1e-6
        for i in range(x.shape[1]):
            xp, xm = x.copy(), x.copy()
            xp[:, i] += h
            xm[:, i] -= h
            fd = (mlp.forward(params, xp)[0][:, j] - mlp.forward(params, xm)[0][:, j]) / (2 * h)
            np.testing.assert_allclose(g[:, i], fd, rtol=1e-6, atol=1e-9)


def test_adam_first_step_moves_by_lr_against_the_sign(small):
    params, x, t, w = small
    _, grads = mlp.backward(params, x, t, w)
    new = mlp.adam(params, grads, {}, lr=1e-3, eps=1e-12)
    for (W, b), (gW, gb), (W1, b1) in zip(params, grads, new):
        np.testing.assert_allclose(W1 - W, -1e-3 * np.sign(gW), atol=1e-9)
        np.testing.assert_allclose(b1 - b, -1e-3 * np.sign(gb), atol=1e-9)


def test_training_reduces_the_loss():
    rng = np.random.default_rng(2)
    params = mlp.init([3, 16, 2], rng)
    x = rng.normal(size=(256, 3))
    t = np.stack([x.sum(1), np.abs(x[:, 0])], 1)
    w = np.ones(2)
    st = {}
    L0 = mlp.loss(params, x, t, w)
    for _ in range(300):
        _, g = mlp.backward(params, x, t, w)
        params = mlp.adam(params, g, st, lr=1e-2)
    assert mlp.loss(params, x, t, w) < 0.1 * L0


# ---------------------------------------------------------------------------


def test_autocall_states_on_hand_made_paths():
    # 2 assets, refs 1; dates t0..t3.  Path 0: called at t2 (worst 1.05);
    # path 1: knocks in at t1 (worst 0.55), never called.
    S = np.array([[[1.0, 1.0], [0.9, 1.2], [1.1, 1.05], [0.5, 0.5]],
                  [[1.0, 1.0], [0.55, 0.9], [0.8, 0.95], [0.7, 0.99]]])
    alive, ki = cv.autocall_states(S, [1.0, 1.0], 1.0, 0.6)
    np.testing.assert_array_equal(alive, [[1, 1, 0], [1, 1, 1]])
    np.testing.assert_array_equal(ki, [[0, 0, 0], [0, 1, 1]])


def _paths(mk, n_paths, seed):
    return np.moveaxis(simulate(mk, seed, 0, np.arange(n_paths)), 1, 2)   # [p, o, i]


def test_hedge_martingale_has_mean_zero_for_any_adapted_hedge():
    mk = Market([1.0, 1.2, 0.8], [0.3, 0.2, 0.25], [[1, .5, .5], [.5, 1, .5], [.5, .5, 1]], 0.03,
                [365, 730, 1095, 1460])
    S = _paths(mk, 1 << 15, 11)
    disc = [mk.disc(o) for o in range(mk.n + 1)]
    # arbitrary, path-dependent but adapted hedge ratios
    delta = np.stack([np.sin(3 * S[:, k, :]) + S[:, :k + 1, :].mean(1) for k in range(mk.n)], 1)
    alive, _ = cv.autocall_states(S, mk.S0, 1.1, 0.6)
    M = cv.hedge_martingale(S, disc, alive, delta)
    assert abs(M.mean()) < 4 * M.std() / math.sqrt(len(M))
    assert M.std() > 0.05


def test_daily_delta_hedge_replicates_a_call():
    """Black-Scholes delta hedging at 250 dates replicates max(S_T - K, 0):
    the hedged payoff's variance is a small fraction of the payoff's."""
    K, sig, r, T = 1.0, 0.2, 0.03, 1.0
    days = list(range(1, 251))
    mk = Market([1.0], [sig], [[1.0]], r, days)
    tau = np.array([0.0] + [dd / 365.0 for dd in days])
    S = _paths(mk, 4096, 5)
    disc = np.exp(-r * tau)
    x = disc[-1] * np.maximum(S[:, -1, 0] - K, 0.0)
    n = len(days)
    delta = np.zeros((len(S), n, 1))
    for k in range(n):
        delta[:, k, 0] = [cf.bs_delta_call(s, K, r, sig, tau[-1] - tau[k]) for s in S[:, k, 0]]
    M = cv.hedge_martingale(S, disc, np.ones((len(S), n), bool), delta)
    y = x - M
    assert y.var() < 0.02 * x.var()
    price = cf.bs_call(1.0, K, r, sig, tau[-1])
    assert abs(y.mean() - price) < 4 * y.std() / math.sqrt(len(y))


def test_multilinear_lookup_is_exact_on_multilinear_functions_and_clamps():
    rng = np.random.default_rng(1)
    G, d = 6, 3
    lo, h = np.array([-1.0, -0.5, 0.2]), np.array([0.4, 0.3, 0.1])
    c = rng.normal(size=8)

    def f(y):
        a, b, e = y[..., 0], y[..., 1], y[..., 2]
        return (c[0] + c[1] * a + c[2] * b + c[3] * e + c[4] * a * b + c[5] * a * e + c[6] * b * e
                + c[7] * a * b * e)
    nodes = np.stack(np.meshgrid(*[lo[i] + h[i] * np.arange(G) for i in range(d)], indexing="ij"), -1)
    table = np.repeat(f(nodes).reshape(-1, 1), d, axis=1) * np.array([1.0, 2.0, -1.0])
    y = lo + h * rng.uniform(0, G - 1, size=(500, d))
    got = cv.table_lookup(table, lo, h, G, y)
    np.testing.assert_allclose(got[:, 0], f(y), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got[:, 1], 2 * f(y), rtol=1e-12, atol=1e-12)
    out = np.array([[-10.0, 0.0 + lo[1], 100.0]])
    clamp = np.array([[lo[0], lo[1], lo[2] + (G - 1) * h[2]]])
    np.testing.assert_allclose(cv.table_lookup(table, lo, h, G, out), cv.table_lookup(table, lo, h, G, clamp))


def test_feature_layout():
    F = cv.autocall_features(np.array([[0.1, -0.2, 0.3]]), np.array([True]), 2, 5,
                             [0.2, 0.25, 0.3], 0.5, 0.03, 1.0, 0.05, 1.0, 0.6)
    np.testing.assert_allclose(F[0], [0.1, -0.2, 0.3, 0.2, 0.25, 0.3, 0.5, 0.03, 1.0, 0.6, 0.4, 1.0,
                                      0.05, 1.0, 0.6, 1.0])


def test_gamma_martingale_has_mean_zero_for_any_adapted_gamma():
    corr = np.array([[1, .5, .3], [.5, 1, .4], [.3, .4, 1]])
    mk = Market([1.0, 1.2, 0.8], [0.3, 0.2, 0.25], corr.tolist(), 0.03, [365, 730, 1095, 1460])
    S = _paths(mk, 1 << 15, 12)
    disc = [mk.disc(o) for o in range(mk.n + 1)]
    tau = [0.0] + [dd / 365.0 for dd in mk.days]
    g = np.stack([np.einsum("pi,pj->pij", np.cos(S[:, k, :]), np.cos(S[:, k, :])) for k in range(mk.n)], 1)
    alive = np.ones((len(S), mk.n), bool)
    M2 = cv.gamma_martingale(S, disc, alive, g, corr, mk.sigma, tau)
    assert abs(M2.mean()) < 4 * M2.std() / math.sqrt(len(M2))
    assert M2.std() > 0.01


def test_quarterly_delta_gamma_hedge_beats_delta_alone():
    """A call hedged at 4 dates with Black-Scholes delta, then with delta and
    gamma (closed-form gamma): the second-order term removes most of what
    the delta hedge leaves."""
    K, sig, r = 1.0, 0.3, 0.02
    days = [91, 182, 273, 365]
    mk = Market([1.0], [sig], [[1.0]], r, days)
    tau = np.array([0.0] + [dd / 365.0 for dd in days])
    S = _paths(mk, 1 << 15, 6)
    disc = np.exp(-r * tau)
    x = disc[-1] * np.maximum(S[:, -1, 0] - K, 0.0)
    n = len(days)
    dl, gm = np.zeros((len(S), n, 1)), np.zeros((len(S), n, 1, 1))
    for k in range(n):
        T = tau[-1] - tau[k]
        s = S[:, k, 0]
        d1 = (np.log(s / K) + (r + 0.5 * sig * sig) * T) / (sig * np.sqrt(T))
        dl[:, k, 0] = [cf.Phi(v) for v in d1]
        # Gamma of the value in today's money: disc_k * bs gamma
        gm[:, k, 0, 0] = np.exp(-0.5 * d1 * d1) / np.sqrt(2 * np.pi) / (s * sig * np.sqrt(T)) / disc[k]
    alive = np.ones((len(S), n), bool)
    M = cv.hedge_martingale(S, disc, alive, dl)
    M2 = cv.gamma_martingale(S, disc, alive, gm, np.array([[1.0]]), [sig], tau)
    v1, v2 = (x - M).var(), (x - M - M2).var()
    assert v2 < 0.6 * v1, (v1, v2)


def test_table_slopes_are_the_derivatives_of_the_interpolant():
    rng = np.random.default_rng(4)
    G, d = 5, 3
    lo, h = np.array([-0.5, 0.0, 0.3]), np.array([0.2, 0.3, 0.1])
    table = rng.normal(size=(G ** d, d))
    y = lo + h * rng.uniform(0.05, G - 1.05, size=(200, d))
    sl = cv.table_slopes(table, lo, h, G, y)
    eps = 1e-6
    for j in range(d):
        yp, ym = y.copy(), y.copy()
        yp[:, j] += eps * h[j]
        ym[:, j] -= eps * h[j]
        fd = (cv.table_lookup(table, lo, h, G, yp) - cv.table_lookup(table, lo, h, G, ym)) / (2 * eps)
        np.testing.assert_allclose(sl[:, :, j], fd, rtol=1e-6, atol=1e-8)


def test_taylor_tables_are_exact_on_affine_functions_and_clamp():
    """Nearest-node Taylor tables: node slopes of an affine table are its
    coefficients (central and one-sided differences alike), and the lookup
    reproduces the affine function anywhere in the grid; points outside
    take the clamped coordinate."""
    G, d = 6, 3
    rng = np.random.default_rng(3)
    A, b = rng.normal(size=(d, d)), rng.normal(size=d)
    lo, h = np.array([-1.0, -0.5, 0.2]), np.array([0.3, 0.2, 0.25])
    nodes = np.stack(np.meshgrid(*[np.arange(G)] * d, indexing="ij"), -1).reshape(-1, d)
    table = nodes @ A.T + b
    sl = cv.node_slopes(table, G)
    np.testing.assert_allclose(sl, np.broadcast_to(A, sl.shape), atol=1e-12)
    y = lo + h * rng.uniform(0.0, G - 1.0, size=(2000, d))
    delta, s = cv.taylor_lookup(table, sl, lo, h, G, y)
    np.testing.assert_allclose(delta, ((y - lo) / h) @ A.T + b, atol=1e-12)
    out = lo + h * np.array([[-2.0, 0.5, G + 3.0]])
    clamp = lo + h * np.array([[0.0, 0.5, G - 1.0]])
    np.testing.assert_allclose(cv.taylor_lookup(table, sl, lo, h, G, out)[0],
                               cv.taylor_lookup(table, sl, lo, h, G, clamp)[0])


def test_taylor_node_slopes_and_nearest_node_on_a_quadratic():
    """On Delta = u^2 along one axis: interior slopes are the exact 2u
    (central differences), the ends one-sided (1 at node 0, 2G - 3 at the
    last), and a point takes its nearest node: u = 2.4 -> node 2 (4 + 4 x
    0.4), u = 2.6 -> node 3 (9 - 6 x 0.4)."""
    G = 7
    table = (np.arange(G, dtype=np.float64) ** 2)[:, None]
    sl = cv.node_slopes(table, G)[:, 0, 0]
    np.testing.assert_allclose(sl, [1.0] + [2.0 * a for a in range(1, G - 1)] + [2.0 * G - 3.0])
    lo, h = np.array([0.0]), np.array([1.0])
    got = cv.taylor_lookup(table, cv.node_slopes(table, G), lo, h, G, np.array([[2.4], [2.6]]))[0][:, 0]
    np.testing.assert_allclose(got, [4.0 + 4.0 * 0.4, 9.0 - 6.0 * 0.4])


def test_taylor_hedges_keep_the_martingales_at_mean_zero():
    """Hedge ratios and gammas from nearest-node Taylor tables (random node
    values) keep E[M] = E[M2] = 0 on GBM paths (a few standard errors)."""
    rng = np.random.default_rng(11)
    N, n, d, G = 200000, 4, 2, 5
    sig = np.array([0.25, 0.3])
    corr = np.array([[1.0, 0.4], [0.4, 1.0]])
    r = 0.02
    tau = np.arange(n + 1) * 0.5
    L = np.linalg.cholesky(corr)
    S = np.ones((N, n + 1, d))
    for k in range(n):
        dt = tau[k + 1] - tau[k]
        z = rng.standard_normal((N, d)) @ L.T
        S[:, k + 1] = S[:, k] * np.exp((r - 0.5 * sig ** 2) * dt + sig * np.sqrt(dt) * z)
    disc = np.exp(-r * tau)
    alive = np.ones((N, n), bool)
    ki = np.zeros((N, n + 1), bool)
    ki[:, 2:] = S[:, 1:2, 0] < 0.9
    lo = np.tile(np.array([-0.6, -0.6]), (n - 1, 1))
    h = np.tile(np.array([0.3, 0.3]), (n - 1, 1))
    tables = rng.normal(0.5, 0.2, size=(n - 1, 2, G ** d, d))
    delta = cv.table_deltas_taylor(S, ki, tables, lo, h, G, [0.5, 0.4])
    M = cv.hedge_martingale(S, disc, alive, delta)
    assert abs(M.mean()) < 4 * M.std() / np.sqrt(N)
    gam = cv.table_gammas_taylor(S, ki, tables, lo, h, G)
    M2 = cv.gamma_martingale(S, disc, alive, gam, corr, sig, tau)
    assert abs(M2.mean()) < 4 * M2.std() / np.sqrt(N)
    assert M.std() > 0.01 and M2.std() > 1e-4


def test_node_records_layout():
    """The engine's 12-float node records: ratios, then s_ij at 3 + 3 i + j."""
    G, d = 4, 2
    rng = np.random.default_rng(5)
    tables = rng.normal(size=(2, 2, G ** d, d))
    rec = cv.node_records(tables, G)
    assert rec.shape == (2, 2, G ** d, 12)
    np.testing.assert_array_equal(rec[..., :d], tables)
    sl = cv.node_slopes(tables[1, 0], G)
    for i in range(d):
        for j in range(d):
            np.testing.assert_array_equal(rec[1, 0, :, 3 + 3 * i + j], sl[:, i, j])
    assert not rec[..., 2].any() and not rec[..., 3 + 3 * 2:].any() and not rec[..., 5].any()
