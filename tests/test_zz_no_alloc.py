"""pc_price_noalloc: pricing without any device allocation.

Some callers cannot allocate GPU memory while they price: code that runs
under an allocator or framework owning all of the device's memory, or code
that must not call cudaMalloc at that point of its run.  pc_price_noalloc
serves them.  It runs the same kernel as pc_price_async but takes its
scratch from a fixed device array of the library.  These tests price
through it twice in a row (the second call reuses the array the first call
left behind) and compare each result with pc_price_async, the entry point
that uses memory the context allocated.  The file is named to be collected
last.
"""
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


def noalloc_sums(eng, m, k, n, seed, offset=0, stream=0):
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    pc.pc_price_noalloc(m, k, n, offset, seed, stream, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("wl,n", [("worst_of_autocall_3u_5d", 1 << 20),
                                  ("daily_barrier_3u_365d", (1 << 16) + 5)])
def test_noalloc_matches_allocating_entry_point_twice(eng, wl, n):
    w = W.ALL[wl]()
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    want = eng.sums(m, k, n, w.seed, 123, 2)
    for _ in range(2):
        got = noalloc_sums(eng, m, k, n, w.seed, 123, 2)
        assert got[2] == n
        np.testing.assert_allclose(got[:2], want[:2], rtol=1e-12, atol=0)


def test_noalloc_rejects_requests_beyond_its_array(eng):
    w = W.european_call()
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError) as ei:
        pc.pc_price_noalloc(m, k, pc.NOALLOC_MAX_PATHS + 1, 0, 1, 0, out.data_ptr())
    assert ei.value.name == "PC_ELIMIT"
    # the largest allowed request still works and matches
    n = pc.NOALLOC_MAX_PATHS
    np.testing.assert_allclose(noalloc_sums(eng, m, k, n, 7)[:2], eng.sums(m, k, n, 7)[:2],
                               rtol=1e-12, atol=0)
