"""Programs that are not streamable in shared memory: the window of
simulated dates in HBM (pc_price with PC_WINDOW_AUTO / PC_WINDOW_HBM).

* where both placements can run, the HBM window gives bit-identical
  per-path payoffs and sums to the shared window;
* an average-rate call summed newest fixing first over 300 daily dates
  (lookback 299, window 512 dates) runs only with the HBM window: per-path
  parity with the oracle, and the shared-only policy refuses it;
* pc_price_info reports the placement and the HBM bytes.
"""
import numpy as np
import pytest

from cases import CASES
from gpu_common import Engine, compare, oracle_paths, torch
import paper_2108_03076_gb300 as pc
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = Engine()
    yield e
    pc.pc_set_window_mode(e.ctx, pc.WINDOW_AUTO)
    e.close()


def reverse_asian_text(n: int, K: float = 1.0) -> str:
    """Average of asset 0 and asset 1 over the n dates ending at $0,
    summed newest fixing first (each term looks back one date further)."""
    T = "(tplus 0 $0)"
    terms = [f"(add (model 0 (tplus {T} {-j})) (model 1 (tplus {T} {-j})))" for j in range(n)]
    s = terms[0]
    for x in terms[1:]:
        s = f"(add {s} {x})"
    return f"(mult (max (sub (div {s} {float(2 * n)}) {K}) 0.0) (payoff {T} 0 1))"


@pytest.mark.parametrize("name", ["autocall", "lookback", "double_barrier", "nested_loops", "basket_and"])
def test_hbm_window_is_bit_identical_to_shared(eng, name):
    text, tp, spec, _ = CASES[name]
    m, k = eng.model(spec), eng.contract(text, tp)
    n, seed = 5000 + 7, 0x1234
    out = {}
    for mode in (pc.WINDOW_SHARED, pc.WINDOW_HBM):
        pc.pc_set_window_mode(eng.ctx, mode)
        info = pc.pc_price_info(m, k, n)
        assert info.hbm_window == (1 if mode == pc.WINDOW_HBM else 0)
        out[mode] = eng.paths(m, k, n, seed)
    pc.pc_set_window_mode(eng.ctx, pc.WINDOW_AUTO)
    np.testing.assert_array_equal(out[pc.WINDOW_SHARED][0], out[pc.WINDOW_HBM][0])
    np.testing.assert_array_equal(out[pc.WINDOW_SHARED][1], out[pc.WINDOW_HBM][1])


def test_long_lookback_program_runs_with_the_hbm_window(eng):
    days = list(range(1, 301))
    spec = W.MarketSpec([1.0, 1.2], [0.25, 0.3], W.const_corr(2, 0.4), 0.02, days)
    text = reverse_asian_text(300, 1.05)
    m, k = eng.model(spec), eng.contract(text, [300])
    pc.pc_set_window_mode(eng.ctx, pc.WINDOW_AUTO)
    info = pc.pc_price_info(m, k, 1 << 20)
    assert info.hbm_window == 1 and info.window == 512
    assert info.hbm_window_bytes == info.grid * info.block * 512 * 2 * 8
    assert info.window_bytes_written_per_path_date == 8
    n, seed = 2048 + 3, 0x77
    x, sums = eng.paths(m, k, n, seed)
    ref, marg = oracle_paths(text, spec, [300], n, seed)
    compare(x, ref, marg, 1.0, "reverse asian")
    assert sums[0] == pytest.approx(x.sum(), rel=1e-9)
    pc.pc_set_window_mode(eng.ctx, pc.WINDOW_SHARED)
    try:
        with pytest.raises(pc.PcError) as e:
            pc.pc_price(m, k, 1000, 1)
        assert e.value.name == "PC_ERANGE"
    finally:
        pc.pc_set_window_mode(eng.ctx, pc.WINDOW_AUTO)
    price, se = pc.pc_price(m, k, 1 << 20, 3)
    assert np.isfinite(price) and se > 0
