"""Pins of the whole oracle pipeline (compile -> paths -> IL semantics ->
average): closed forms, Gauss-Hermite quadrature over the oracle's own
normals-to-payoff map, and exact expectation on small binomial trees against
hand-written payoff functions."""
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import cl, closed_forms as cf, contracts as C, il, il_text, mc, paths
from oracle.paths import Market


def market(spec) -> Market:
    return Market(**vars(spec))


def within(est, want, k=3.0):
    assert abs(est.price - want) <= k * est.stderr, (est.price, want, est.stderr)


def test_european_call_2p16_paths_against_black_scholes():
    w = W.european_call()
    est = mc.price(il_text.parse(w.il_text), market(w.market), {"$0": 1}, 0, 1, w.n_paths, w.seed)
    want = cf.bs_call(100.0, 100.0, 0.03, 0.2, 1.0)
    assert want == pytest.approx(9.413403383853016, rel=1e-14)
    within(est, want)
    # discounted payoff sd 14.11 -> relative SE 0.586% at 2^16 paths
    assert est.stderr / est.price == pytest.approx(0.00586, rel=0.05)


def test_digital_forward_zero_coupon_put_call_parity():
    mk = Market([100.0], [0.2], [[1.0]], 0.03, [365])
    d = {"T": 1}
    n, seed = 1 << 15, 77
    dig = mc.price(cl.compile_contr(C.digital_cl(100.0)), mk, d, 0, 1, n, seed)
    within(dig, cf.digital_call(100, 100, 0.03, 0.2, 1.0))
    assert cf.digital_call(100, 100, 0.03, 0.2, 1.0) == pytest.approx(0.5045722918443936, rel=1e-14)
    fwd = mc.price(cl.compile_contr(C.forward_cl(100.0)), mk, d, 0, 1, n, seed)
    within(fwd, cf.forward(100, 100, 0.03, 1.0))
    zcb = mc.price(cl.compile_contr(C.zero_coupon_cl()), mk, d, 0, 1, n, seed)
    # constant payoff: exact up to the rounding of the path-ordered sums
    assert zcb.price == pytest.approx(0.9704455335485082, rel=1e-12) and zcb.stderr < 1e-8
    # call - put = forward path by path (same draws)
    call = cl.compile_contr(C.european_cl(100.0))
    put = cl.compile_contr(cl.Translate(C.T, cl.Scale(
        cl.op("max", cl.op("sub", cl.RLit(100.0), cl.Obs(0, 0)), cl.RLit(0.0)), C.xfer())))
    x_c = mc.payoffs(call, mk, d, 0, 1, 4096, seed)
    x_p = mc.payoffs(put, mk, d, 0, 1, 4096, seed)
    x_f = mc.payoffs(cl.compile_contr(C.forward_cl(100.0)), mk, d, 0, 1, 4096, seed)
    np.testing.assert_allclose(x_c - x_p, x_f, atol=1e-12)
    # reversed parties negate the value
    x_rev = mc.payoffs(call, mk, d, 1, 0, 4096, seed)
    np.testing.assert_array_equal(x_rev, -x_c)


def test_exchange_option_against_margrabe():
    mk = Market([100.0, 95.0], [0.25, 0.3], [[1, 0.5], [0.5, 1]], 0.03, [182, 365])
    est = mc.price(cl.compile_contr(C.exchange_cl()), mk, {"T": 2}, 0, 1, 1 << 16, 31)
    within(est, cf.margrabe(100.0, 95.0, 0.25, 0.3, 0.5, 1.0))


def test_gauss_hermite_three_dates():
    """E[payoff] by tensor Gauss-Hermite over the three normals of a 3-date,
    1-underlying path, through the oracle's own map normals -> path -> IL
    value; Monte Carlo must land within 3 SE."""
    mk = Market([1.0], [0.25], [[1.0]], 0.02, [120, 240, 365])
    # Asian-style call on the 3-date average plus a leg paying S - 1.1 on the
    # first date S >= 1.1 (continuous in the normals, so the quadrature
    # converges: 48 and 64 nodes per axis agree to 3e-4, below one SE)
    c = cl.Both(
        cl.Translate(cl.TNum(3), cl.Scale(cl.op("max", cl.op("sub", cl.op("div", cl.op(
            "add", cl.op("add", cl.Obs(0, 0), cl.Obs(0, -1)), cl.Obs(0, -2)), cl.RLit(3.0)),
            cl.RLit(1.0)), cl.RLit(0.0)), C.xfer())),
        cl.Translate(cl.TNum(1), cl.IfWithin(cl.ge(cl.Obs(0, 0), cl.RLit(1.1)), cl.TNum(2),
                                             cl.Scale(cl.op("sub", cl.Obs(0, 0), cl.RLit(1.1)), C.xfer()),
                                             cl.Zero())))
    prog = cl.compile_contr(c)
    x, w = np.polynomial.hermite_e.hermegauss(48)
    w = w / math.sqrt(2 * math.pi)
    Z = np.array(list(itertools.product(x, repeat=3)))               # [node, j]
    Wt = np.prod(np.array(list(itertools.product(w, repeat=3))), axis=1)
    S = paths.simulate_from_normals(mk, Z[:, :, None])
    args = il.Args(rho=mc.env_from_paths(mk, S), delta={}, now=0, d=mk.disc, p1=0, p2=1)
    gh = float((il.evaluate(prog, args, idx=np.arange(len(Z))) * Wt).sum())
    est = mc.price(prog, mk, {}, 0, 1, 1 << 16, 5)
    within(est, gh)


def _crr_paths(S0, sigma, r, days):
    """All 2^n paths of a Cox-Ross-Rubinstein tree on the grid, with their
    risk-neutral probabilities; ordinal 0 is the spot."""
    tau = np.concatenate([[0.0], np.asarray(days, float) / 365.0])
    dts = np.diff(tau)
    out, probs = [], []
    for moves in itertools.product([0, 1], repeat=len(days)):
        s, pr, path = S0, 1.0, [S0]
        for mv, dt in zip(moves, dts):
            u = math.exp(sigma * math.sqrt(dt))
            q = (math.exp(r * dt) - 1 / u) / (u - 1 / u)
            s = s * (u if mv else 1 / u)
            pr *= q if mv else 1 - q
            path.append(s)
        out.append(path)
        probs.append(pr)
    return np.array(out), np.array(probs)


def _tree_args(S, mk):
    return il.Args(rho=lambda l, t, idx: S[idx, t], delta={"T": mk.n}, now=0, d=mk.disc,
                   p1=0, p2=1)


def test_binomial_autocall_against_hand_written_payoff():
    """3-date, 1-underlying version of the autocall note, every path of a CRR
    tree: compiled IL value == the payoff written directly from the term
    sheet (call at k if S_k/S0 >= 1 paying 1 + 0.05k; else at maturity S_3/S0
    if any S_k/S0 <= 0.6, else 1), each discounted at its payment date."""
    mk = Market([1.0], [0.45], [[1.0]], 0.03, [365, 730, 1095])
    S, pr = _crr_paths(1.0, 0.45, 0.03, mk.days)
    prog = cl.compile_contr(C.autocall_cl([1.0], n_dates=3))
    got = il.evaluate(prog, _tree_args(S, mk), idx=np.arange(len(S)))

    def by_hand(s):
        for k in (1, 2, 3):
            if s[k] / 1.0 >= 1.0:
                return (1 + 0.05 * k) * mk.disc(k)
        ki = any(s[k] <= 0.6 for k in (1, 2, 3))
        return (s[3] if ki else 1.0) * mk.disc(3)

    want = np.array([by_hand(s) for s in S])
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-15)
    assert (got * pr).sum() == pytest.approx((want * pr).sum(), rel=1e-14)
    assert len(set(np.round(want, 12))) >= 4          # several distinct outcomes


def test_binomial_barrier_against_hand_written_payoff():
    mk = Market([1.0], [0.5], [[1.0]], 0.01, [1, 2, 3, 4])
    S, pr = _crr_paths(1.0, 0.5, 0.01, mk.days)
    S = S * np.array([1.0, 1.0, 0.9, 0.8, 0.7])[None, :]   # make the barrier reachable
    prog = cl.compile_contr(C.daily_barrier_cl([1.0], barrier=0.8, n_spreads=4, top=1.6))
    got = il.evaluate(prog, _tree_args(S, mk), idx=np.arange(len(S)))

    def by_hand(s):
        if any(s[k] <= 0.8 for k in range(0, 5)):
            return 0.0
        w = s[4]
        return min(max(w, 0.0), 1.6) * mk.disc(4)

    np.testing.assert_allclose(got, [by_hand(s) for s in S], rtol=1e-14, atol=1e-15)
