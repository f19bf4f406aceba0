"""Failure detection, tested without a GPU fault.

* PC_ETIMEOUT: a context limit far below a finite launch's run time; the
  call returns the error, the work completes on the stream, and the context
  prices correctly afterwards.
* PC_ENOMEM: injected allocation failures (no allocator call) in the
  context's scratch growth, model tables, contract upload and portfolio
  plan; nothing leaks and the next calls succeed.
* PC_EDEVICE: the device status word raised as a clamping kernel would;
  the next blocking call reports it and the one after is clean.
* The tensor-core product's bounded waits: with the producer withholding
  its first copies, the waits expire after about 10 ms, the kernel returns
  and the network's next blocking call reports PC_ETIMEOUT; after that the
  network computes the same gradients as before.
"""
import numpy as np
import pytest

from gpu_common import torch
import paper_2108_03076_gb300 as pc
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03076_gb300 import build
    build.build()
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    c = pc.pc_create(0, s.cuda_stream)
    yield c
    pc.pc_destroy(c)


def objects(c, w):
    spec = w.market
    m = pc.pc_model_create(c, spec.S0, spec.sigma, spec.corr, spec.r, spec.days)
    words, consts = pc.pc_assemble(w.il_text)
    return m, pc.pc_load_payoff(c, words, consts, w.tparams, 0, 1)


def test_timeout_returns_and_context_recovers(ctx):
    w = W.daily_barrier()                      # 2^22 paths x 365 dates: ~9 ms on the device
    m, k = objects(ctx, w)
    try:
        want = pc.pc_price(m, k, 1 << 16, 7)
        pc.pc_set_timeout(ctx, 1e-4)
        with pytest.raises(pc.PcError) as ei:
            pc.pc_price(m, k, w.n_paths, w.seed)
        assert ei.value.name == "PC_ETIMEOUT"
        pc.pc_set_timeout(ctx, 300.0)
        assert pc.pc_price(m, k, 1 << 16, 7) == want
        with pytest.raises(pc.PcError):
            pc.pc_set_timeout(ctx, 0.0)
    finally:
        pc.pc_contract_destroy(k)
        pc.pc_model_destroy(m)


def test_injected_allocation_failures(ctx):
    w = W.daily_barrier()
    spec = w.market
    words, consts = pc.pc_assemble(w.il_text)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # model tables
    pc.pc_debug_fail_allocations(ctx, 1)
    with pytest.raises(pc.PcError) as ei:
        pc.pc_model_create(ctx, spec.S0, spec.sigma, spec.corr, spec.r, spec.days)
    assert ei.value.name == "PC_ENOMEM"
    m = pc.pc_model_create(ctx, spec.S0, spec.sigma, spec.corr, spec.r, spec.days)
    # contract upload
    pc.pc_debug_fail_allocations(ctx, 1)
    with pytest.raises(pc.PcError) as ei:
        pc.pc_load_payoff(ctx, words, consts, w.tparams, 0, 1)
    assert ei.value.name == "PC_ENOMEM"
    k = pc.pc_load_payoff(ctx, words, consts, w.tparams, 0, 1)
    try:
        want = pc.pc_price(m, k, 1 << 12, 3)
        # growth of the tile-partial scratch (2^22 paths need more than the first buffer)
        pc.pc_debug_fail_allocations(ctx, 1)
        with pytest.raises(pc.PcError) as ei:
            pc.pc_price(m, k, 1 << 22, 3)
        assert ei.value.name == "PC_ENOMEM"
        # portfolio plan
        pc.pc_debug_fail_allocations(ctx, 1)
        with pytest.raises(pc.PcError) as ei:
            pc.pc_price_batch([m, m], [k, k], [4096, 4096], 5)
        assert ei.value.name == "PC_ENOMEM"
        pc.pc_debug_fail_allocations(ctx, 0)
        assert pc.pc_price(m, k, 1 << 12, 3) == want
        big = pc.pc_price(m, k, 1 << 22, 3)
        assert np.isfinite(big[0])
    finally:
        pc.pc_contract_destroy(k)
        pc.pc_model_destroy(m)
    torch.cuda.synchronize()
    # what the context still holds (its grown scratch) is below 256 MiB; the
    # failed calls held nothing
    assert free0 - torch.cuda.mem_get_info()[0] < (256 << 20)


def test_device_status_word_reports_edevice(ctx):
    w = W.european_call()
    m, k = objects(ctx, w)
    try:
        want = pc.pc_price(m, k, 1 << 14, 9)
        pc.pc_debug_set_status(ctx, 1)
        with pytest.raises(pc.PcError) as ei:
            pc.pc_price(m, k, 1 << 14, 9)
        assert ei.value.name == "PC_EDEVICE"
        assert pc.pc_price(m, k, 1 << 14, 9) == want
    finally:
        pc.pc_contract_destroy(k)
        pc.pc_model_destroy(m)


def test_tensor_core_bounded_wait_expiry(ctx):
    widths = [16, 256, 256, 256, 5]
    net = pc.pc_mlp_create(ctx, widths, 1024, seed=3)
    try:
        if not pc.pc_mlp_gemm_info(net):
            pytest.skip("tcgen05 products not available")
        rng = np.random.default_rng(2)
        n = 512
        x = torch.tensor(rng.normal(size=(n, 16)).astype(np.float32), device="cuda")
        t = torch.tensor(rng.normal(size=(n, 5)).astype(np.float32), device="cuda")
        w = np.ones(5, np.float32)
        g0 = torch.empty(pc.pc_mlp_query(net).n_params, dtype=torch.float32, device="cuda")
        loss0 = pc.pc_mlp_gradients(net, x.data_ptr(), t.data_ptr(), w, n, g0.data_ptr())
        y = torch.empty((n, 5), dtype=torch.float32, device="cuda")
        pc.pc_debug_mlp_withhold_tma(net, True)
        pc.pc_mlp_forward(net, x.data_ptr(), n, y.data_ptr())   # every product's waits expire
        pc.pc_debug_mlp_withhold_tma(net, False)
        g1 = torch.empty_like(g0)
        with pytest.raises(pc.PcError) as ei:
            pc.pc_mlp_gradients(net, x.data_ptr(), t.data_ptr(), w, n, g1.data_ptr())
        assert ei.value.name == "PC_ETIMEOUT"
        # the status word was cleared: the network works as before
        loss1 = pc.pc_mlp_gradients(net, x.data_ptr(), t.data_ptr(), w, n, g1.data_ptr())
        assert loss1 == loss0
        assert torch.equal(g0, g1)
    finally:
        pc.pc_mlp_destroy(net)


def test_fused_table_build_bounded_wait_expiry(ctx):
    """The one-launch hedge-table build (cv_tables_tc) with its producer
    withholding the first weight chunk: every bounded wait expires (about
    10 ms), the kernel returns, pc_cv_tables reports PC_ETIMEOUT; afterwards
    the same build gives the tables it gave before, bit for bit."""
    from paper_2108_03076_gb300 import learned_cv as L
    w = W.worst_of_autocall()
    s = w.market
    model = pc.pc_model_create(ctx, s.S0, s.sigma, s.corr, s.r, s.days)
    net = L.LearnedCV(ctx, seed=5)
    try:
        if not pc.pc_mlp_gemm_info(net.net):
            pytest.skip("tcgen05 products not available")
        _, t0 = net.tables(model)
        ref = t0.cpu().numpy().copy()
        pc.pc_debug_mlp_withhold_tma(net.net, True)
        with pytest.raises(pc.PcError) as ei:
            net.tables(model, out=t0)
        assert ei.value.name == "PC_ETIMEOUT"
        pc.pc_debug_mlp_withhold_tma(net.net, False)
        _, t1 = net.tables(model, out=t0)
        n = pc.pc_cv_table_size(pc.pc_cv_grid(model, 12, 4.5))
        np.testing.assert_array_equal(t1.cpu().numpy()[:n].view(np.uint32), ref[:n].view(np.uint32))
    finally:
        net.close()
        pc.pc_model_destroy(model)
