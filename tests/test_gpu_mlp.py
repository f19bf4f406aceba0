"""GPU network kernels (pc_mlp_*) against the oracle's FP64 network,
element by element.

The oracle runs on the same BF16-rounded weights and inputs.  The device
stores every hidden activation and every back-propagated signal in BF16
(relative rounding <= 2^-9 per stored value), accumulates products in FP32
and evaluates softplus with the SFU.  Each element is checked against

    |g - r| <= c 2^-8 (|r| + s)

with r the oracle's value and s the scale of its layer:
* outputs: s = RMS of the output layer's term sizes |W_L| |h_{L-1}| + |b_L|
  (a stored activation's 2^-9 reaches an output through one product with
  exact BF16 weights: error ~ 2^-9 s), c = 2;
* gradients: s = RMS of the layer's oracle gradient, c = 8 (a gradient
  element is a sum of products of two stored values, 2 x 2^-9, plus the
  propagated roundings of the signals above it: the loss signal and one
  stored signal per layer, 2^-9 each, four layers: 2^-8 (1 + 2) relative to
  the terms; the terms' RMS exceeds the gradient's RMS where the sum
  cancels, hence 8).
A numpy model of these roundings stays within 0.22 (outputs) and 3.8
(gradients) of the respective bounds' c 2^-8 (|r| + s) / c, on the shapes
tested here.  A wrong sign then fails on every element above s / 63, a
wrong index or transposed operand everywhere.
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


def assert_close_el(got, want, c, scale, what):
    """Element-wise |got - want| <= c 2^-8 (|want| + scale)."""
    tol = c * 2.0 ** -8 * (np.abs(want) + scale)
    bad = np.abs(got - want) > tol
    assert not bad.any(), (what, int(bad.sum()), got[bad][:4], want[bad][:4], tol[bad][:4])


def output_scale(params, x):
    """RMS of the output layer's term sizes |W_L| |h_{L-1}| + |b_L|."""
    _, cache = mlp.forward(params, x)
    W, b = params[-1]
    return float(np.sqrt(np.mean((np.abs(cache[-1][0]) @ np.abs(W).T + np.abs(b)) ** 2)))


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
        assert_close_el(y, ref, 2.0, output_scale(rounded(params), bf16(x)), "output")
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
            assert_close_el(gW, rW, 8.0, np.sqrt(np.mean(rW ** 2)), f"dW{l}")
            assert_close_el(gb, rb, 8.0, np.sqrt(np.mean(rb ** 2)), f"db{l}")
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
        sc = output_scale(rounded(params), bf16(x))
        tc, ws = outs
        assert np.isfinite(tc).all()
        assert_close_el(tc, ref, 2.0, sc, "tcgen05 output")
        assert_close_el(ws, ref, 2.0, sc, "mma.sync output")
        # the two kernels differ only by FP32 summation order (and the BF16
        # rounding of hidden activations it can flip)
        assert rel_err(tc, ws) < 5e-3, rel_err(tc, ws)
    finally:
        pc.pc_mlp_destroy(net)


@pytest.mark.parametrize("widths,n", [(WIDTHS, 4099), ([16, 1024, 384, 5], 2000), ([9, 128, 64], 200)])
def test_tensor_core_gradients_match_oracle_and_warp_kernel(ctx, widths, n):
    """tcgen05 backward products: the data gradient reads W N-major, the
    weight gradient reads dZ M-major and the layer input N-major (TMA boxes
    of 64 x 64 in the MN-major swizzled layout), split over the rows in
    64-row chunks with a fixed-order sum.  Element by element against the
    oracle's FP64 backpropagation, and against the warp-level kernel (same
    BF16 operands, FP32 sums in another order)."""
    rng = np.random.default_rng(n + 3 * len(widths))
    params = mlp.init(widths, rng)
    net = pc.pc_mlp_create(ctx, widths, 4160)
    try:
        assert pc.pc_mlp_gemm_info(net), "tcgen05 products not available"
        pc.pc_mlp_set_params(net, flat(params))
        x = rng.normal(size=(n, widths[0])).astype(np.float32)
        t = rng.normal(size=(n, widths[-1])).astype(np.float32)
        w = np.linspace(0.25, 2.0, widths[-1]).astype(np.float32)
        dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        outs = []
        for kind in (pc.MLP_GEMM_AUTO, pc.MLP_GEMM_MMA_SYNC):
            pc.pc_mlp_set_gemm(net, kind)
            dg = torch.full((pc.pc_mlp_query(net).n_params,), float("nan"), dtype=torch.float32, device="cuda")
            pc.pc_mlp_gradients(net, dx.data_ptr(), dt.data_ptr(), w, n, dg.data_ptr())
            torch.cuda.synchronize()
            outs.append(unflat(dg.double().cpu().numpy(), widths))
        _, grads = mlp.backward(rounded(params), bf16(x), t.astype(np.float64), w.astype(np.float64))
        for l, ((tW, tb), (sW, sb), (rW, rb)) in enumerate(zip(outs[0], outs[1], grads)):
            assert np.isfinite(tW).all() and np.isfinite(tb).all(), l
            assert_close_el(tW, rW, 8.0, np.sqrt(np.mean(rW ** 2)), f"tcgen05 dW{l}")
            assert_close_el(tb, rb, 8.0, np.sqrt(np.mean(rb ** 2)), f"tcgen05 db{l}")
            assert_close_el(sW, rW, 8.0, np.sqrt(np.mean(rW ** 2)), f"mma.sync dW{l}")
            assert rel_err(tW, sW) < 1e-2, (l, rel_err(tW, sW))
    finally:
        pc.pc_mlp_destroy(net)


def test_tensor_core_products_on_a_65536_row_batch(ctx):
    """A 2^16-row gradient (every product on tcgen05: forward, data and
    weight gradients) agrees with the warp-level kernel's element by element
    to FP32 summation order, and the forward outputs too."""
    rng = np.random.default_rng(65536)
    n = 1 << 16
    params = mlp.init(WIDTHS, rng)
    net = pc.pc_mlp_create(ctx, WIDTHS, n)
    try:
        assert pc.pc_mlp_gemm_info(net), "tcgen05 products not available"
        pc.pc_mlp_set_params(net, flat(params))
        x = rng.normal(size=(n, 16)).astype(np.float32)
        t = rng.normal(size=(n, 5)).astype(np.float32)
        w = np.array([1.0, 0.5, 0.25, 2.0, 1.0], np.float32)
        dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        grads, ys = [], []
        for kind in (pc.MLP_GEMM_AUTO, pc.MLP_GEMM_MMA_SYNC):
            pc.pc_mlp_set_gemm(net, kind)
            dg = torch.empty(pc.pc_mlp_query(net).n_params, dtype=torch.float32, device="cuda")
            for _ in range(3):
                pc.pc_mlp_gradients(net, dx.data_ptr(), dt.data_ptr(), w, n, dg.data_ptr())
            dy = torch.empty((n, 5), dtype=torch.float32, device="cuda")
            pc.pc_mlp_forward(net, dx.data_ptr(), n, dy.data_ptr())
            torch.cuda.synchronize()
            grads.append(unflat(dg.double().cpu().numpy(), WIDTHS))
            ys.append(dy.double().cpu().numpy())
        assert_close_el(ys[0], ys[1], 2.0, float(np.sqrt(np.mean(ys[1] ** 2))), "output")
        for l, ((tW, tb), (sW, sb)) in enumerate(zip(*grads)):
            assert np.isfinite(tW).all(), l
            # both are FP32 sums of the same BF16 products: within the
            # gradient rule of the oracle comparisons, element by element
            assert_close_el(tW, sW, 8.0, np.sqrt(np.mean(sW ** 2)), f"dW{l}")
            assert_close_el(tb, sb, 8.0, np.sqrt(np.mean(sb ** 2)), f"db{l}")
    finally:
        pc.pc_mlp_destroy(net)


def test_tensor_core_training_matches_warp_kernel(ctx):
    """The training step with every product on tcgen05 fits like the
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


def test_adam_step_matches_oracle(ctx):
    """One training step from set parameters: the device gathers its
    minibatch with Philox (counter (row, 0, step, 0), key = seed, word 0,
    index mod n_data), computes the gradient and takes an Adam step.  The
    oracle's Adam step on the device's gradient of the same rows (from
    pc_mlp_gradients) gives the new parameters element by element, to FP32
    rounding."""
    from oracle.paths import philox4x32_10, split_seed
    rng = np.random.default_rng(5)
    params = mlp.init(WIDTHS, rng)
    n_data, batch, seed, lr = 3001, 512, 0x0123456789ABCDEF, 1e-3
    x = rng.normal(size=(n_data, 16)).astype(np.float32)
    t = rng.normal(size=(n_data, 5)).astype(np.float32)
    w = np.array([1.0, 0.5, 0.25, 2.0, 1.0], np.float32)
    rows = np.arange(batch, dtype=np.uint64)
    idx = (philox4x32_10([rows, np.uint64(0), np.uint64(0), np.uint64(0)], split_seed(seed))[0]
           % np.uint64(n_data)).astype(np.int64)
    net = pc.pc_mlp_create(ctx, WIDTHS, 1024)
    try:
        p0 = flat(params)
        pc.pc_mlp_set_params(net, p0)
        xg, tg = torch.tensor(x[idx], device="cuda"), torch.tensor(t[idx], device="cuda")
        dg = torch.empty(pc.pc_mlp_query(net).n_params, dtype=torch.float32, device="cuda")
        pc.pc_mlp_gradients(net, xg.data_ptr(), tg.data_ptr(), w, batch, dg.data_ptr())
        g = unflat(dg.double().cpu().numpy(), WIDTHS)
        pc.pc_mlp_set_params(net, p0)     # also clears the Adam moments and the step count
        dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        pc.pc_mlp_train(net, dx.data_ptr(), dt.data_ptr(), n_data, w, batch, 1, lr, seed)
        got = pc.pc_mlp_get_params(net).astype(np.float64)
        want = flat(mlp.adam(unflat(p0.astype(np.float64), WIDTHS), g, {}, lr)).astype(np.float64)
        # the same step on the oracle's own gradient differs only where the
        # gradient is within its rounding of zero (Adam's first step is
        # lr * g / (|g| + eps): a sign)
        assert np.max(np.abs(got - want) - (2e-6 * lr + 2.0 ** -22 * np.abs(want))) <= 0, \
            np.max(np.abs(got - want))
        moved = np.abs(got - p0) > 0.5 * lr
        assert moved.mean() > 0.9
    finally:
        pc.pc_mlp_destroy(net)
