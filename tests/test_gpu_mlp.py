"""GPU network kernels (pc_mlp_*) against the oracle's FP64 network.

The oracle runs on the same BF16-rounded weights and inputs; the device
stores every activation and back-propagated signal in BF16 (relative
rounding <= 2^-9 per stored value) and accumulates in FP32, so outputs and
gradients agree to a few 2^-9 relative (bounds below, with margin).
"""
import numpy as np
import pytest

from gpu_common import torch
import paper_2108_03076_gb300 as pc
from oracle import mlp

pytestmark = pytest.mark.gpu

WIDTHS = [16, 256, 256, 256, 5]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03076_gb300 import build
    build.build()
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    c = pc.pc_create(0, st.cuda_stream)
    yield c
    pc.pc_destroy(c)


def bf16(a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().double().numpy()


def flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def unflat(v, widths):
    out, k = [], 0
    for fin, fout in zip(widths[:-1], widths[1:]):
        W = v[k:k + fin * fout].reshape(fout, fin)
        k += fin * fout
        b = v[k:k + fout]
        k += fout
        out.append((W, b))
    return out


def rounded(params):
    # the device multiplies with BF16 weights; biases stay FP32
    return [(bf16(W), np.asarray(b, np.float32).astype(np.float64)) for W, b in params]


def rel_err(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("n", [1, 64, 1000, 4099])
def test_forward_matches_oracle(ctx, n):
    rng = np.random.default_rng(n)
    params = mlp.init(WIDTHS, rng)
    net = pc.pc_mlp_create(ctx, WIDTHS, 2048)
    try:
        pc.pc_mlp_set_params(net, flat(params))
        np.testing.assert_array_equal(pc.pc_mlp_get_params(net), flat(params))
        x = rng.normal(size=(n, 16)).astype(np.float32)
        dx = torch.tensor(x, device="cuda")
        dy = torch.empty((n, 5), dtype=torch.float32, device="cuda")
        pc.pc_mlp_forward(net, dx.data_ptr(), n, dy.data_ptr())
        torch.cuda.synchronize()
        y = dy.double().cpu().numpy()
        ref, _ = mlp.forward(rounded(params), bf16(x))
        assert rel_err(y, ref) < 1.5e-2, rel_err(y, ref)
        assert np.abs(y - ref).max() < 5e-2 * np.abs(ref).max() + 1e-3
    finally:
        pc.pc_mlp_destroy(net)


@pytest.mark.parametrize("n", [64, 777, 2048])
def test_gradients_match_oracle(ctx, n):
    rng = np.random.default_rng(100 + n)
    params = mlp.init(WIDTHS, rng)
    net = pc.pc_mlp_create(ctx, WIDTHS, 2048)
    try:
        pc.pc_mlp_set_params(net, flat(params))
        x = rng.normal(size=(n, 16)).astype(np.float32)
        t = rng.normal(size=(n, 5)).astype(np.float32)
        w = np.array([1.0, 0.5, 0.25, 2.0, 0.0], np.float32)
        dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        dg = torch.empty(pc.pc_mlp_query(net).n_params, dtype=torch.float32, device="cuda")
        loss = pc.pc_mlp_gradients(net, dx.data_ptr(), dt.data_ptr(), w, n, dg.data_ptr())
        L, grads = mlp.backward(rounded(params), bf16(x), t.astype(np.float64), w.astype(np.float64))
        assert loss == pytest.approx(L, rel=1e-2)
        got = unflat(dg.double().cpu().numpy(), WIDTHS)
        for l, ((gW, gb), (rW, rb)) in enumerate(zip(got, grads)):
            assert rel_err(gW, rW) < 3e-2, (l, rel_err(gW, rW))
            assert rel_err(gb, rb) < 3e-2, (l, rel_err(gb, rb))
        # the output with weight 0 receives no gradient
        np.testing.assert_array_equal(got[-1][0][4], 0.0)
        assert got[-1][1][4] == 0.0
    finally:
        pc.pc_mlp_destroy(net)


def test_training_fits_and_is_deterministic(ctx):
    rng = np.random.default_rng(9)
    n = 1 << 14
    x = rng.uniform(-1, 1, size=(n, 16)).astype(np.float32)
    t = np.stack([x[:, :4].sum(1), np.sin(2 * x[:, 0]), x[:, 1] * x[:, 2], np.maximum(x[:, 3], 0),
                  np.zeros(n)], 1).astype(np.float32)
    w = np.array([1, 1, 1, 1, 0], np.float32)
    dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    runs = []
    for _ in range(2):
        net = pc.pc_mlp_create(ctx, WIDTHS, 1024, seed=3)
        try:
            first = pc.pc_mlp_train(net, dx.data_ptr(), dt.data_ptr(), n, w, 512, 1, 1e-3, 77)
            last = pc.pc_mlp_train(net, dx.data_ptr(), dt.data_ptr(), n, w, 512, 1500, 1e-3, 77)
            assert pc.pc_mlp_query(net).steps == 1501
            runs.append(pc.pc_mlp_get_params(net))
        finally:
            pc.pc_mlp_destroy(net)
        assert last < 0.05 * first, (first, last)
    np.testing.assert_array_equal(runs[0], runs[1])


@pytest.mark.parametrize("widths,n", [(WIDTHS, 13825), ([16, 1024, 384, 5], 4099), ([9, 128, 64], 200)])
def test_tensor_core_forward_matches_oracle_and_warp_kernel(ctx, widths, n):
    """tcgen05 forward products (TMA-staged, TMEM accumulators) on the
    table-build size (13,825 rows: 109 row tiles, the last one ragged), a
    deep K (1024: sixteen 64-deep chunks through the four-stage ring) and
    narrow layers (N = 64 tiles), against the oracle and the warp-level
    kernel (same BF16 operands, FP32 sums in another order)."""
    rng = np.random.default_rng(n + len(widths))
    params = mlp.init(widths, rng)
    net = pc.pc_mlp_create(ctx, widths, 16384)
    try:
        assert pc.pc_mlp_gemm_info(net), "tcgen05 products not available"
        pc.pc_mlp_set_params(net, flat(params))
        x = rng.normal(size=(n, widths[0])).astype(np.float32)
        dx = torch.tensor(x, device="cuda")
        outs = []
        for kind in (pc.MLP_GEMM_AUTO, pc.MLP_GEMM_MMA_SYNC):
            pc.pc_mlp_set_gemm(net, kind)
            dy = torch.full((n, widths[-1]), float("nan"), dtype=torch.float32, device="cuda")
            pc.pc_mlp_forward(net, dx.data_ptr(), n, dy.data_ptr())
            torch.cuda.synchronize()
            outs.append(dy.double().cpu().numpy())
        assert not pc.pc_mlp_gemm_info(net)
        ref, _ = mlp.forward(rounded(params), bf16(x))
        tc, ws = outs
        assert np.isfinite(tc).all()
        assert rel_err(tc, ref) < 1.5e-2, rel_err(tc, ref)
        assert np.abs(tc - ref).max() < 5e-2 * np.abs(ref).max() + 1e-3
        # the two kernels differ only by FP32 summation order (and the BF16
        # rounding of hidden activations it can flip)
        assert rel_err(tc, ws) < 5e-3, rel_err(tc, ws)
    finally:
        pc.pc_mlp_destroy(net)


def test_tensor_core_training_matches_warp_kernel(ctx):
    """The training step with tcgen05 forward products fits like the
    warp-level kernel's and is deterministic."""
    rng = np.random.default_rng(19)
    n = 1 << 13
    x = rng.uniform(-1, 1, size=(n, 16)).astype(np.float32)
    t = np.stack([x[:, :4].sum(1), np.sin(2 * x[:, 0]), x[:, 1] * x[:, 2], np.maximum(x[:, 3], 0),
                  np.zeros(n)], 1).astype(np.float32)
    w = np.array([1, 1, 1, 1, 0], np.float32)
    dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    res = {}
    for kind, rep in ((pc.MLP_GEMM_AUTO, 0), (pc.MLP_GEMM_AUTO, 1), (pc.MLP_GEMM_MMA_SYNC, 0)):
        net = pc.pc_mlp_create(ctx, WIDTHS, 1024, seed=3)
        try:
            pc.pc_mlp_set_gemm(net, kind)
            first = pc.pc_mlp_train(net, dx.data_ptr(), dt.data_ptr(), n, w, 512, 1, 1e-3, 77)
            last = pc.pc_mlp_train(net, dx.data_ptr(), dt.data_ptr(), n, w, 512, 800, 1e-3, 77)
            res[kind, rep] = (first, last, pc.pc_mlp_get_params(net))
        finally:
            pc.pc_mlp_destroy(net)
    np.testing.assert_array_equal(res[pc.MLP_GEMM_AUTO, 0][2], res[pc.MLP_GEMM_AUTO, 1][2])
    f_tc, l_tc, _ = res[pc.MLP_GEMM_AUTO, 0]
    f_ws, l_ws, _ = res[pc.MLP_GEMM_MMA_SYNC, 0]
    assert f_tc == pytest.approx(f_ws, rel=1e-2)
    assert l_tc < 0.1 * f_tc and l_ws < 0.1 * f_ws
    assert l_tc == pytest.approx(l_ws, rel=0.5)
