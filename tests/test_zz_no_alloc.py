"""pc_price_noalloc: pricing without any device allocation.

Some callers cannot allocate GPU memory while they price: code that runs
under an allocator or framework owning all of the device's memory, or code
that must not call cudaMalloc at that point of its run.  pc_price_noalloc
serves them.  It runs the same kernel as pc_price_async but takes its
scratch from a fixed device array of the library, whose address pc_create
looks up.  These tests price through it twice in a row (the second call
reuses the array the first call left behind) and compare each result with
pc_price_async, the entry point that uses memory the context allocated:
the two run the same kernel on the same inputs, so the sums are equal bit
for bit.  One test makes the first call of a fresh context through
pc_price_noalloc and checks that the device's free memory did not move.
The file is named to be collected last.
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


def noalloc_sums(m, k, n, seed, offset=0, stream=0):
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
        got = noalloc_sums(m, k, n, w.seed, 123, 2)
        assert got[2] == n
        assert np.array_equal(got[:2], want[:2]), (got, want)


def test_noalloc_first_call_on_a_fresh_context_takes_no_device_memory():
    """A fresh context whose first pricing call is pc_price_noalloc: the
    device's free memory is the same before and after the call (a device
    allocation moves it by at least its 2 MiB granularity), and the sums
    equal pc_price_async's afterwards."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.ALL["worst_of_autocall_3u_5d"]()
    s = torch.cuda.Stream()
    ctx = pc.pc_create(0, s.cuda_stream)
    spec = w.market
    m = pc.pc_model_create(ctx, spec.S0, spec.sigma, spec.corr, spec.r, spec.days)
    words, consts = pc.pc_assemble(w.il_text)
    k = pc.pc_load_payoff(ctx, words, consts, w.tparams, 0, 1)
    try:
        n = 1 << 20
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            pc.pc_price_noalloc(m, k, n, 0, w.seed, 0, out.data_ptr())
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy()
        ref = torch.zeros(4, dtype=torch.float64, device="cuda")
        pc.pc_price_async(m, k, n, 0, w.seed, 0, ref.data_ptr())
        torch.cuda.synchronize()
        assert got[2] == n and np.array_equal(got[:2], ref.cpu().numpy()[:2])
    finally:
        pc.pc_contract_destroy(k)
        pc.pc_model_destroy(m)
        pc.pc_destroy(ctx)


def test_noalloc_refuses_windows_beyond_shared_memory(eng):
    """A program that looks back 300 dates keeps its window of dates in HBM
    under pc_price_async; pc_price_noalloc keeps windows in shared memory
    only and refuses it with PC_ERANGE."""
    w = W.ALL["reverse_asian_2u_300d"]()
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError) as ei:
        pc.pc_price_noalloc(m, k, 4096, 0, w.seed, 0, out.data_ptr())
    assert ei.value.name == "PC_ERANGE"
    assert eng.sums(m, k, 4096, w.seed)[2] == 4096


def test_noalloc_rejects_requests_beyond_its_array(eng):
    w = W.european_call()
    m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError) as ei:
        pc.pc_price_noalloc(m, k, pc.NOALLOC_MAX_PATHS + 1, 0, 1, 0, out.data_ptr())
    assert ei.value.name == "PC_ELIMIT"
    # the largest allowed request still works and matches
    n = pc.NOALLOC_MAX_PATHS
    assert np.array_equal(noalloc_sums(m, k, n, 7)[:2], eng.sums(m, k, n, 7)[:2])
