"""GPU host-side paths of the API: the per-context compile cache keyed by
the compiler's inputs, program uploads through the two-half pinned staging
buffer under many back-to-back loads, contracts freed in stream order, and
hedge-table builds replayed from their captured graph.

Each check compares against a fresh context (nothing cached) or against
the same call made the other way, value for value."""
import numpy as np
import pytest

from gpu_common import Engine, torch
import paper_2108_03076_gb300 as pc
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    yield e
    e.close()


def fresh_sums(spec, text, tparams, p1, p2, n, seed):
    """(sum, sumsq, n) from a context of its own (empty caches)."""
    cur = torch.cuda.current_stream()
    e = Engine()
    try:
        m = e.model(spec)
        k = e.contract(text, tparams, p1, p2)
        return e.sums(m, k, n, seed)
    finally:
        e.close()
        torch.cuda.set_stream(cur)


def test_compile_cache_keys_on_every_input(eng):
    """Loading one bytecode with other template parameters or parties gives
    the program of those inputs, not a cached one."""
    spec = W.MarketSpec([100.0], [0.2], [[1.0]], 0.03, list(range(1, 366)))
    text = W.barrier_ladder_text([100.0])
    m = eng.model(spec)
    got = {}
    for tp, p1, p2 in [([365], 0, 1), ([180], 0, 1), ([365], 1, 0), ([365], 0, 1), ([180], 0, 1)]:
        k = eng.contract(text, tp, p1, p2)
        got.setdefault((tuple(tp), p1, p2), []).append(eng.sums(m, k, 1 << 14, 9))
    for key, runs in got.items():
        for r in runs[1:]:
            np.testing.assert_array_equal(r, runs[0])
        np.testing.assert_array_equal(runs[0], fresh_sums(spec, text, list(key[0]), key[1], key[2], 1 << 14, 9))
    assert not np.array_equal(got[((365,), 0, 1)][0], got[((180,), 0, 1)][0])
    assert got[((365,), 1, 0)][0][0] == pytest.approx(-got[((365,), 0, 1)][0][0], rel=1e-12)


def test_many_loads_through_the_staging_buffer(eng):
    """Three thousand programs loaded back to back (the staging halves wrap
    about a hundred times), then a sample priced: every program is its
    own, as a fresh context loads it."""
    items = W.portfolio(n_contracts=64)
    spec_models = [eng.model(it.market) for it in items]
    loaded = []
    for rep in range(47):
        for i, it in enumerate(items):
            w, k = pc.pc_assemble(it.il_text)
            loaded.append((i, pc.pc_load_payoff(eng.ctx, w, k, it.tparams, 0, 1)))
    try:
        rng = np.random.default_rng(3)
        for j in rng.choice(len(loaded), 12, replace=False):
            i, k = loaded[j]
            it = items[i]
            got = eng.sums(spec_models[i], k, 4096, 21 + i)
            want = fresh_sums(it.market, it.il_text, it.tparams, 0, 1, 4096, 21 + i)
            np.testing.assert_array_equal(got, want)
    finally:
        for _, k in loaded:
            pc.pc_contract_destroy(k)


def test_table_build_replays_equal_fresh_builds(eng):
    """A hedge-table build replayed from its captured graph (same buffer)
    equals the first build, a build into another buffer, and a build by a
    second network with the same parameters."""
    from paper_2108_03076_gb300 import learned_cv as LCV
    w = W.worst_of_autocall()
    m = eng.model(w.market)
    net = LCV.LearnedCV(eng.ctx, seed=11)
    net2 = LCV.LearnedCV(eng.ctx, seed=12)
    try:
        pc.pc_mlp_set_params(net2.net, pc.pc_mlp_get_params(net.net))
        def used(t):  # 16-byte node groups: the first d = 3 words are written
            return t.cpu().numpy().reshape(-1, 4)[:, :3].copy()

        d1, t1 = net.tables(m, grid=8)
        first = used(t1)
        for _ in range(3):
            d1, t1 = net.tables(m, grid=8, out=t1)
            np.testing.assert_array_equal(used(t1), first)
        d2, t2 = net.tables(m, grid=8)
        np.testing.assert_array_equal(used(t2), first)
        d3, t3 = net2.tables(m, grid=8)
        np.testing.assert_array_equal(used(t3), first)
        assert [d1.delta0[i] for i in range(3)] == [d3.delta0[i] for i in range(3)]
        assert np.isfinite(first).all() and np.abs(first).max() > 0
    finally:
        net.close()
        net2.close()
