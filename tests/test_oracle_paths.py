"""Pins of the oracle's path generator: Philox4x32-10 against cuRAND's host
generator, uniforms, Box-Muller special values and moments, the Brownian
bridge covariance, the Cholesky factor and GBM moments."""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

from oracle import paths
from oracle.paths import Market


def _curand():
    for cand in ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]:
        if cand and os.path.exists(cand) or (cand and not cand.startswith("/")):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    return None


CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def curand_host_philox(seed: int, offset: int, n_words: int) -> np.ndarray:
    """n_words 32-bit outputs of cuRAND's CPU-side Philox4x32-10 generator."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = np.zeros(n_words, dtype=np.uint32)
        assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(n_words)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return buf


@pytest.mark.parametrize("seed,offset", [(0x123456789ABCDEF0, 0), (0xDEADBEEF0BADF00D, 1 << 34),
                                         (42, 3 << 50), (0xFFFFFFFFFFFFFFFF, 4 * 70001)])
def test_philox_matches_curand_host_generator(seed, offset):
    """cuRAND's host generator emits block q = offset/4 + b from counter
    (low and high words of q >> 16, q & 0xFFFF, 0) under key (seed_lo, seed_hi)
    -- a layout observed on this toolkit; 2^17 blocks are compared, which
    exercises counter words 0, 1, 2 and the key schedule."""
    nblk = 1 << 17
    got = curand_host_philox(seed, offset, 4 * nblk).reshape(nblk, 4)
    q = np.arange(nblk, dtype=np.uint64) + np.uint64(offset // 4)
    hi = q >> np.uint64(16)
    x = paths.philox4x32_10([hi & np.uint64(0xFFFFFFFF), hi >> np.uint64(32),
                             q & np.uint64(0xFFFF), np.uint64(0)], paths.split_seed(seed))
    want = np.stack([v.astype(np.uint32) for v in x], axis=1)
    np.testing.assert_array_equal(want, got)


def test_philox_output_statistics():
    n = 1 << 18
    ctr = np.arange(n, dtype=np.uint64)
    x = paths.philox4x32_10([ctr, np.uint64(7), np.uint64(0), np.uint64(3)], (1, 2))
    w = np.concatenate([v for v in x]).astype(np.uint64)
    bits = np.unpackbits(w.astype(np.uint32).view(np.uint8))
    assert abs(bits.mean() - 0.5) < 5 * 0.5 / math.sqrt(len(bits))
    counts = np.bincount((w >> np.uint64(24)).astype(np.int64), minlength=256)
    e = len(w) / 256
    chi2 = ((counts - e) ** 2 / e).sum()
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    # every counter word and the key change the output
    base = [np.uint64(5), np.uint64(6), np.uint64(7), np.uint64(8)]
    y0 = [int(v) for v in paths.philox4x32_10(base, (9, 10))]
    for k in range(4):
        c = list(base)
        c[k] = np.uint64(int(c[k]) ^ 1)
        assert [int(v) for v in paths.philox4x32_10(c, (9, 10))] != y0
    assert [int(v) for v in paths.philox4x32_10(base, (9, 11))] != y0


def test_u24_is_exact_odd_multiple_of_2_pow_minus_25():
    x = np.array([0, 255, 256, 0xFFFFFFFF, 0x80000000], dtype=np.uint64)
    u = paths.u24(x)
    np.testing.assert_array_equal(u, [2.0 ** -25, 2.0 ** -25, 3 * 2.0 ** -25,
                                      1.0 - 2.0 ** -25, 0.5 + 2.0 ** -25])
    k = u * 2.0 ** 25
    assert np.all(k == np.round(k)) and np.all(k % 2 == 1)


def test_box_muller_special_values():
    ua = np.array([math.exp(-0.5), math.exp(-0.5), math.exp(-2.0), 0.5])
    ub = np.array([0.0, 0.25, 0.5, 0.125])
    z0, z1 = paths.box_muller(ua, ub)
    r = np.sqrt(-2 * np.log(ua))
    np.testing.assert_allclose(r, [1.0, 1.0, 2.0, math.sqrt(2 * math.log(2))], rtol=1e-15)
    np.testing.assert_allclose(z0, [1.0, 0.0, -2.0, math.sqrt(math.log(2))], atol=1e-15)
    np.testing.assert_allclose(z1, [0.0, 1.0, 0.0, math.sqrt(math.log(2))], atol=1e-15)


def test_normals_moments_and_independence():
    z = paths.normals(0x5EED, 0, np.arange(1 << 14, dtype=np.uint64), 64)
    v = z.reshape(-1)
    n = len(v)
    assert abs(v.mean()) < 5 / math.sqrt(n)
    assert abs(v.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs((v ** 4).mean() - 3) < 5 * math.sqrt(96 / n)
    c = np.corrcoef(z[:, :8].T)
    assert np.abs(c - np.eye(8)).max() < 5 / math.sqrt(z.shape[0])


def test_normal_index_layout():
    """normal m of a path is output word m & 3 of counter (m >> 2, p_lo, p_hi, stream)."""
    seed, stream, p = 0xABCDEF0123, 5, np.array([2 ** 33 + 17], dtype=np.uint64)
    z = paths.normals(seed, stream, p, 12)[0]
    for m in range(12):
        x = paths.philox4x32_10([np.uint64(m >> 2), np.uint64(17), np.uint64(2), np.uint64(stream)],
                                paths.split_seed(seed))
        pair = (m & 3) // 2
        ua, ub = paths.u24(x[2 * pair]), paths.u24(x[2 * pair + 1])
        zz = paths.box_muller(ua, ub)[m & 1]
        assert z[m] == zz


def _walk_order(nodes, n):
    """The nodes in the order a walk producing dates 1..n in turn computes
    them, by brute force: the walk holds the set of dates whose W is known;
    to produce date t it takes the nearest known date r above t and
    computes the node whose interval is (t - 1, r), then repeats with that
    node's date, until t itself is known."""
    by_interval = {(nd.l, nd.r): j for j, nd in enumerate(nodes) if nd.r >= 0}
    root = [j for j, nd in enumerate(nodes) if nd.r < 0][0]
    known, order = {0}, []
    for t in range(1, n + 1):
        if t not in known and not [x for x in known if x > t]:
            order.append(root)
            known.add(n)
        while t not in known:
            r = min(x for x in known if x > t)
            j = by_interval[(t - 1, r)]
            order.append(j)
            known.add(nodes[j].m)
    return order


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 31, 100, 365])
def test_generation_order_is_the_date_ordered_walk(n):
    """generation_order ranks the nodes in the order a date-by-date walk
    computes them (checked against the walk itself); with d normals per node
    in that order, node k takes normals d k .. d k + d - 1."""
    nodes = paths.bridge_schedule(np.arange(n + 1) / 365.0)
    order = _walk_order(nodes, n)
    assert sorted(order) == list(range(n))
    rank = paths.generation_order(nodes)
    assert [int(rank[j]) for j in order] == list(range(n))
    p = np.array([3, 2 ** 32 + 9], dtype=np.uint64)
    for d in (1, 2, 3, 4):
        z = paths.node_normals(nodes, d, 0xBEEF, 2, p)
        flat = paths.normals(0xBEEF, 2, p, n * d)
        for k, j in enumerate(order):
            assert np.array_equal(z[:, j, :], flat[:, d * k:d * k + d])


@pytest.mark.parametrize("days", [[365], [100, 365], [1, 2, 3, 4, 5], list(range(1, 366)),
                                  [7, 30, 31, 90, 200, 201, 364, 900], list(range(10, 3651, 10))])
def test_bridge_covariance_is_min_of_times(days):
    """The bridge maps iid normals to W with Cov(W_s, W_t) = min(s, t): the
    matrix B of the linear map z -> W satisfies B B^T = [min(tau_i, tau_j)]."""
    tau = np.concatenate([[0.0], np.asarray(days, float) / 365.0])
    n = len(days)
    nodes = paths.bridge_schedule(tau)
    assert sorted(nd.m for nd in nodes) == list(range(1, n + 1))
    assert nodes[0].m == n
    B = paths.bridge_apply(nodes, np.eye(n), n)[:, 1:].T          # [date, normal]
    np.testing.assert_allclose(B @ B.T, np.minimum.outer(tau[1:], tau[1:]), rtol=0, atol=1e-13)


def test_bridge_bfs_order():
    nodes = paths.bridge_schedule(np.arange(9) / 8.0)
    assert [nd.m for nd in nodes] == [8, 4, 2, 6, 1, 3, 5, 7]
    nodes = paths.bridge_schedule(np.arange(6) / 5.0)
    assert [nd.m for nd in nodes] == [5, 2, 1, 3, 4]


def test_cholesky_pairwise_half():
    mk = Market([1, 1, 1], [0.2] * 3, [[1, .5, .5], [.5, 1, .5], [.5, .5, 1]], 0.0, [365])
    L = mk.cholesky()
    want = np.array([[1, 0, 0], [.5, math.sqrt(.75), 0], [.5, .25 / math.sqrt(.75), math.sqrt(2 / 3)]])
    np.testing.assert_allclose(L, want, atol=1e-15)
    np.testing.assert_allclose(L @ L.T, np.asarray(mk.corr, float), atol=1e-14)


def test_gbm_moments_and_correlation():
    mk = Market([100.0, 50.0], [0.2, 0.3], [[1, 0.6], [0.6, 1]], 0.03, [91, 182, 365])
    n = 1 << 16
    S = paths.simulate(mk, 123, 0, np.arange(n))
    tau = mk.tau()
    for i in range(2):
        for o in range(1, 4):
            m = S[:, i, o].mean()
            se = S[:, i, o].std() / math.sqrt(n)
            assert abs(m - mk.S0[i] * math.exp(mk.r * tau[o])) < 4 * se
    lr = np.log(S[:, :, 3] / S[:, :, 2])
    c = np.corrcoef(lr.T)[0, 1]
    assert abs(c - 0.6) < 5 * (1 - 0.36) / math.sqrt(n)
    # independent increments: consecutive log-returns uncorrelated
    l1 = np.log(S[:, 0, 2] / S[:, 0, 1])
    l2 = np.log(S[:, 0, 3] / S[:, 0, 2])
    assert abs(np.corrcoef(l1, l2)[0, 1]) < 5 / math.sqrt(n)
    assert np.all(S[:, :, 0] == np.asarray(mk.S0)[None, :])
