// pc_cv_api.cpp -- pc_cv_* / pc_price_cv: table grids from the model, the
// network evaluation at the table nodes, and the control-variate launch.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "pc_cv.h"
#include "pc_handles.h"
#include "pc_mlp.h"

using namespace pc;

extern "C" pc_status pc_mlp_query(const pc_mlp *net, pc_mlp_info *info);
extern "C" pc_status pc_mlp_forward(pc_mlp *net, const float *d_x, size_t n, float *d_y);

namespace {

size_t nodes_of(const pc_cv_desc *c) {
  size_t v = 1;
  for (int i = 0; i < c->d; ++i) v *= size_t(c->grid);
  return v;
}

pc_status check_desc(const pc_model *m, const pc_cv_desc *c) {
  if (!m || !c) return fail(PC_EINVAL, "null argument");
  if (c->d != m->H.d || c->n != m->H.n) return fail(PC_EINVAL, "control-variate description does not match the model");
  if (c->d < 1 || c->d > kCvMaxD || c->n < 1 || c->n > kCvMaxDates)
    return fail(PC_ELIMIT, "control variate: d must be 1..3 and n 1..32");
  if (c->grid < 2 || c->grid > 64) return fail(PC_EINVAL, "grid must be 2..64");
  for (int k = 0; k + 1 < c->n; ++k)
    for (int i = 0; i < c->d; ++i)
      if (!(c->h[k][i] > 0.f)) return fail(PC_EINVAL, "table spacing must be positive");
  for (int i = 0; i < c->d; ++i)
    if (!(c->ref[i] > 0.f)) return fail(PC_EINVAL, "reference levels must be positive");
  return PC_OK;
}

CvArgs device_args(const pc_cv_desc *c, const float *tables, const ModelHost &H, bool pilot) {
  CvArgs a;
  std::memset(&a, 0, sizeof(a));
  a.tables = tables;
  a.d = c->d;
  a.n = c->n;
  a.grid = c->grid;
  a.nodes = int32_t(nodes_of(c));
  for (int i = 0; i < 3; ++i) {
    a.ref[i] = c->ref[i];
    a.delta0[i] = c->delta0[i];
  }
  if (c->delta0_on_device && tables)  // after the tables (pc_cv_tables_async)
    a.delta0_dev = tables + size_t(std::max(0, c->n - 1)) * 2 * nodes_of(c) * kCvRecord;
  a.call_level = c->call_level;
  a.ki_level = c->ki_level;
  a.coupon = c->coupon;
  std::memcpy(a.lo, c->lo, sizeof(a.lo));
  std::memcpy(a.h, c->h, sizeof(a.h));
  for (int k = 0; k < kCvMaxDates; ++k)
    for (int i = 0; i < kCvMaxD; ++i) {
      const double h = c->h[k][i] > 0.f ? double(c->h[k][i]) : 1.0;
      a.ua[k][i] = float(std::log(2.0) / h);
      a.ub[k][i] = float(double(c->lo[k][i]) / h);
      a.inv_h[k][i] = float(1.0 / h);
    }
  // closed-form second moments of the discounted returns per period
  for (int k = 0; k < std::min(H.n, kCvMaxDates); ++k) {
    const double dt = double(H.tau[k + 1]) - double(H.tau[k]);
    for (int i = 0; i < H.d && i < kCvMaxD; ++i)
      for (int j = 0; j < H.d && j < kCvMaxD; ++j)
        a.cq[k][i * kCvMaxD + j] =
            float(std::expm1(H.corr[size_t(i) * H.d + j] * H.sigma[i] * H.sigma[j] * dt));
  }
  for (int i = 0; i < kCvMaxD; ++i) a.inv_ref[i] = c->ref[i] > 0.f ? float(1.0 / double(c->ref[i])) : 0.f;
  a.beta = c->beta;
  a.beta2 = c->use_gamma ? c->beta2 : 0.f;
  a.use_gamma = c->use_gamma ? 1 : 0;
  a.pilot = pilot ? 1 : 0;
  return a;
}

// The control-variate pricing launch.  The hedge gains accumulate as the
// evaluator generates each date, so the launch keeps the program's own
// window of dates (in registers for a specialised kernel when that window is
// one date).
pc_status cv_launch(const pc_model *m, const pc_contract *k, const pc_cv_desc *c, const float *tables,
                    uint64_t n_paths, uint64_t seed, double *d_out, float *d_xm, bool pilot) {
  pc_status s = check_desc(m, c);
  if (s != PC_OK) return s;
  if (!tables && c->n > 1) return fail(PC_EINVAL, "null tables");
  if (reinterpret_cast<uintptr_t>(tables) & 15u) return fail(PC_EINVAL, "tables must be 16-byte aligned");
  Launch L;
  s = prepare(m, k, n_paths, 0, seed, 0, L);
  if (s != PC_OK) return s;
  pc_ctx *ctx = m->ctx;
  const Layout lay = L.args.lay;
  const size_t pool = (k->prog.pool.size() + 3) & ~size_t(3);
  int block = 0, best = 0;
  size_t smem = 0;
  for (int b = kBlock; b >= 32; b /= 2) {
    const size_t sm = price_smem_bytes(k->prog.code.size(), pool, lay.words, b);
    if (sm + kStaticSmemReserve > size_t(ctx->max_smem)) continue;
    const int warps = cv_blocks_per_sm(c->d, b, sm, device_args(c, tables, m->H, pilot)) * (b / 32);
    if (warps > best) { best = warps; block = b; smem = sm; }
  }
  if (!block) return fail(PC_ELIMIT, "program + per-path state with the control variate exceed shared memory");
  PriceArgs a = L.args;
  a.lay = lay;
  a.width = pilot ? 8 : 4;
  reduction_chunks(a.n_tiles, a.chunk_tiles, a.n_chunks);
  s = ensure_partials(ctx, size_t(a.n_tiles) * size_t(a.width));
  if (s != PC_OK) return s;
  a.tile_partials = ctx->d_partials;
  a.control = ctx->d_control;
  a.out = d_out;
  a.out_paths = d_xm;
  CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  const CvArgs ca = device_args(c, tables, m->H, pilot);
  if (ctx->jit && jit_eligible(k)) {
    // the contract's run-time specialised control-variate kernel: the
    // evaluator keeps its operand stack in registers, so the stack words
    // leave the per-thread shared region
    const bool win_regs = lay.win == 1;
    cudaKernel_t jk = nullptr;
    // register bound: 5 resident blocks by default (measured at 2^22 paths
    // of the autocall: 4 / 5 / 6 blocks 0.428 / 0.396 / 0.392 ms first
    // order, 0.490 / 0.466 / 0.552 ms with the second-order term)
    s = jit_kernel(k, m->H.d, kJitCv + cv_mode(d_xm != nullptr, ca) + (win_regs ? kCvWinRegs : 0), kBlock, jk,
                   ctx->cv_min_blocks > 0 ? ctx->cv_min_blocks : kJitCvMinBlocks);
    if (s != PC_OK) return s;
    const void *kern = reinterpret_cast<const void *>(jk);
    Layout &jl = a.lay;
    const int shift = jl.off_bstack;
    jl.stack = 0;
    jl.off_bstack -= shift;
    jl.off_cache -= shift;
    jl.off_win -= shift;
    jl.words -= shift;
    if (win_regs) jl.words = jl.off_win;  // the frontier's S in registers: no window words
    const size_t jsm = price_smem_bytes(k->prog.code.size(), pool, jl.words, kBlock);
    int nb = 0;
    CU(jit_occupancy(ctx, kern, kBlock, jsm, nb), "jit occupancy");
    if (nb < 1) return fail(PC_ELIMIT, "specialised control-variate kernel cannot be resident");
    const uint64_t jneed = (a.n_tiles + kBlock / 32 - 1) / (kBlock / 32);
    const int jgrid = int(std::min<uint64_t>(uint64_t(ctx->sm_count) * nb, jneed));
    CvArgs cv = ca;
    void *args[] = {&a, &cv};
    CU(cudaLaunchKernel(kern, dim3(jgrid), dim3(kBlock), args, jsm, ctx->stream),
       "specialised control-variate kernel");
    return PC_OK;
  }
  const uint64_t need = (a.n_tiles + block / 32 - 1) / (block / 32);
  const int grid = int(std::min<uint64_t>(uint64_t(ctx->sm_count) * best / (block / 32), need));
  CU(launch_cv(a, ca, grid, block, smem, ctx->stream), "control-variate kernel");
  return PC_OK;
}

}  // namespace

extern "C" {

pc_status pc_cv_labels(size_t n, int32_t d, const double *prices, const double *spots, double bump,
                       int32_t width, float *out) {
  if (!prices || !spots || !out) return fail(PC_EINVAL, "null argument");
  if (d < 1 || d > PC_MAX_UNDERLYINGS || width < 1 + d) return fail(PC_EINVAL, "need 1 <= d <= 4 and width >= 1 + d");
  if (!(bump > 0.0)) return fail(PC_EINVAL, "bump must be > 0");
  for (size_t c = 0; c < n; ++c) {
    float *row = out + c * size_t(width);
    row[0] = float(prices[c]);
    for (int i = 0; i < d; ++i) {
      const double up = prices[(1 + 2 * size_t(i)) * n + c], dn = prices[(2 + 2 * size_t(i)) * n + c];
      row[1 + i] = float((up - dn) / (2.0 * bump * spots[c * size_t(d) + i]));
    }
    for (int j = 1 + d; j < width; ++j) row[j] = 0.f;
  }
  return PC_OK;
}

pc_status pc_cv_grid(const pc_model *m, int32_t grid, float width_sd, pc_cv_desc *c) {
  if (!m || !c) return fail(PC_EINVAL, "null argument");
  if (m->H.d > kCvMaxD || m->H.n > kCvMaxDates) return fail(PC_ELIMIT, "control variate: d <= 3, n <= 32");
  if (grid < 2 || grid > 64 || !(width_sd > 0.f)) return fail(PC_EINVAL, "grid 2..64, width_sd > 0");
  const ModelHost &H = m->H;
  c->d = H.d;
  c->n = H.n;
  c->grid = grid;
  c->beta = 1.f;
  c->beta2 = 1.f;
  c->use_gamma = 0;
  for (int k = 1; k < H.n; ++k) {
    const double tau = double(H.tau[k]);
    for (int i = 0; i < 3; ++i) {
      if (i < H.d) {
        const double sg = H.sigma[i], mid = std::log(H.S0[i]) + (H.r - 0.5 * sg * sg) * tau;
        const double half = double(width_sd) * sg * std::sqrt(tau);
        c->lo[k - 1][i] = float(mid - half);
        c->h[k - 1][i] = float(2.0 * half / (grid - 1));
      } else {
        c->lo[k - 1][i] = 0.f;
        c->h[k - 1][i] = 1.f;
      }
    }
  }
  return PC_OK;
}

pc_status pc_cv_table_size(const pc_cv_desc *c, size_t *floats) {
  if (!c || !floats) return fail(PC_EINVAL, "null argument");
  if (c->d < 1 || c->d > 3 || c->n < 1 || c->grid < 2) return fail(PC_EINVAL, "bad description");
  *floats = size_t(std::max(0, c->n - 1)) * 2 * nodes_of(c) * kCvRecord;
  return PC_OK;
}

}  // extern "C"

namespace {
// The table build (pc_cv_tables; with `async`, pc_cv_tables_async).
pc_status cv_tables(pc_mlp *net, const pc_model *m, pc_cv_desc *c, float *d_tables, size_t cap, bool async) {
  pc_status s = check_desc(m, c);
  if (s != PC_OK) return s;
  pc_mlp_info info;
  s = pc_mlp_query(net, &info);
  if (s != PC_OK) return s;
  if (info.widths[0] != kCvFeatures || info.widths[info.n_layers] != kCvOutputs)
    return fail(PC_EINVAL, "network must map 16 inputs to 5 outputs");
  size_t need = 0;
  pc_cv_table_size(c, &need);
  if (cap < need + (async ? 4 : 0) || ((need || async) && !d_tables)) return fail(PC_EINVAL, "table capacity too small");
  if (reinterpret_cast<uintptr_t>(d_tables) & 15u) return fail(PC_EINVAL, "tables must be 16-byte aligned");
  const ModelHost &H = m->H;
  CvFeatureArgs fa;
  std::memset(&fa, 0, sizeof(fa));
  for (int i = 0; i < H.d; ++i) {
    fa.ln_spot[i] = float(std::log(H.S0[i]));
    fa.sigma[i] = float(H.sigma[i]);
  }
  fa.rho = H.d > 1 ? float(H.corr[1]) : 0.f;
  fa.r = float(H.r);
  for (int o = 0; o <= H.n; ++o) fa.tau[o] = H.tau[o];
  const size_t rows = need / kCvRecord + 1;
  pc_ctx *ctx = m->ctx;
  CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  float *buf = mlp_scratch(net, rows * (kCvFeatures + kCvOutputs) + 64);
  if (!buf) return fail(PC_ENOMEM, "table scratch");
  float *X = buf, *Y = buf + rows * kCvFeatures, *d0 = async ? d_tables + need : Y + rows * kCvOutputs;
  const CvArgs ca = device_args(c, nullptr, m->H, false);
  float *pin = mlp_pinned(net);
  if (pin) {
    // the whole build (features, forward, scatter, read-back of delta0 and
    // the network's status) as one CUDA graph, captured once per set of
    // arguments and replayed
    // (the pricing-only fields -- betas, the second-order switch, delta0,
    // which this call outputs -- do not enter the features kernel)
    CvArgs kc = ca;
    kc.beta = kc.beta2 = 0.f;
    kc.use_gamma = kc.pilot = 0;
    for (float &v : kc.delta0) v = 0.f;
    std::vector<uint8_t> key(sizeof(kc) + sizeof(fa) + 4 * sizeof(uint64_t));
    const uint64_t extra[4] = {reinterpret_cast<uint64_t>(d_tables), reinterpret_cast<uint64_t>(buf), rows,
                               async ? 1u : 0u};
    std::memcpy(key.data(), &kc, sizeof(kc));
    std::memcpy(key.data() + sizeof(ca), &fa, sizeof(fa));
    std::memcpy(key.data() + sizeof(ca) + sizeof(fa), extra, sizeof(extra));
    cudaGraphExec_t *slot = mlp_graph(net, key);
    if (!*slot) {
      cudaStream_t cap = nullptr;
      CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
      cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      pc_status st = PC_OK;
      if (e == cudaSuccess) {
        CvTablesTc tt;
        if (mlp_cv_tables_tc(net, rows, d_tables, d0, tt)) {
          // one launch: features, every layer on tcgen05, scatter
          e = launch_cv_tables_tc(tt, kc, fa, cap);
        } else {
          e = launch_cv_features(kc, fa, X, rows, cap);
          if (e == cudaSuccess) st = mlp_forward_on(net, X, rows, Y, cap);
          if (e == cudaSuccess && st == PC_OK) e = launch_cv_scatter(Y, kCvOutputs, rows, c->d, d_tables, d0, cap);
        }
        if (e == cudaSuccess && st == PC_OK) e = launch_cv_slopes(d_tables, rows - 1, kc.nodes, c->grid, c->d, cap);
        if (e == cudaSuccess && st == PC_OK && !async)
          e = cudaMemcpyAsync(pin, d0, 4 * sizeof(float), cudaMemcpyDeviceToHost, cap);
        if (e == cudaSuccess && st == PC_OK && !async)
          e = cudaMemcpyAsync(pin + 4, mlp_status_word(net), sizeof(int32_t), cudaMemcpyDeviceToHost, cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess && st == PC_OK) e = cudaGraphInstantiate(slot, graph, 0);
        if (graph) cudaGraphDestroy(graph);
      }
      cudaStreamDestroy(cap);
      if (st != PC_OK) return st;
      if (e != cudaSuccess) {
        *slot = nullptr;
        return cuda_fail(e, "table-build graph");
      }
    }
    CU(cudaGraphLaunch(*slot, ctx->stream), "table build");
    if (async) {
      c->delta0_on_device = 1;
      for (float &v : c->delta0) v = 0.f;
      return PC_OK;
    }
    s = wait_stream(ctx);
    if (s != PC_OK) return s;
    int32_t status = 0;
    std::memcpy(&status, pin + 4, sizeof(status));
    if (status != 0) return mlp_status(net);  // clears the word, reports PC_ETIMEOUT
    for (int i = 0; i < 3; ++i) c->delta0[i] = i < c->d ? pin[i] : 0.f;
    c->delta0_on_device = 0;
    return PC_OK;
  }
  cudaError_t e = launch_cv_features(ca, fa, X, rows, ctx->stream);
  if (e != cudaSuccess) s = cuda_fail(e, "table features");
  if (s == PC_OK) s = pc_mlp_forward(net, X, rows, Y);
  if (s == PC_OK) {
    e = launch_cv_scatter(Y, kCvOutputs, rows, c->d, d_tables, d0, ctx->stream);
    if (e == cudaSuccess) e = launch_cv_slopes(d_tables, rows - 1, ca.nodes, c->grid, c->d, ctx->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "table scatter");
  }
  float h0[4] = {0, 0, 0, 0};
  if (s == PC_OK && !async) {
    e = cudaMemcpyAsync(h0, d0, 4 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "delta0 copy");
  }
  if (s == PC_OK) s = mlp_status(net);
  if (s != PC_OK) return s;
  for (int i = 0; i < 3; ++i) c->delta0[i] = i < c->d ? h0[i] : 0.f;
  c->delta0_on_device = async ? 1 : 0;
  return PC_OK;
}
}  // namespace

extern "C" {

pc_status pc_cv_tables(pc_mlp *net, const pc_model *m, pc_cv_desc *c, float *d_tables, size_t cap) {
  return cv_tables(net, m, c, d_tables, cap, false);
}

pc_status pc_cv_tables_async(pc_mlp *net, const pc_model *m, pc_cv_desc *c, float *d_tables, size_t cap) {
  return cv_tables(net, m, c, d_tables, cap, true);
}

// Sums of the launch (width doubles) to the host, with the status check.
pc_status cv_sums(pc_ctx *ctx, int width, double *h) {
  double st[5];
  CU(cudaMemcpyAsync(h, ctx->d_gout, size_t(width) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
     "result copy");
  CU(cudaMemcpyAsync(st, ctx->d_res, 5 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "status copy");
  pc_status s = wait_stream(ctx);
  if (s != PC_OK) return s;
  int32_t status;
  std::memcpy(&status, &st[4], 4);
  return check_status(ctx, status);
}

pc_status pc_price_cv(const pc_model *m, const pc_contract *k, const pc_cv_desc *c, const float *d_tables,
                      uint64_t n_paths, uint64_t seed, double *out) {
  if (!out) return fail(PC_EINVAL, "null output");
  if (n_paths < 2) return fail(PC_EINVAL, "n_paths must be >= 2 for a standard error");
  if (!m) return fail(PC_EINVAL, "null model");
  pc_ctx *ctx = m->ctx;
  pc_status s = cv_launch(m, k, c, d_tables, n_paths, seed, ctx->d_gout, nullptr, false);
  if (s != PC_OK) return s;
  double h[4];
  s = cv_sums(ctx, 4, h);
  if (s != PC_OK) return s;
  const double N = double(n_paths);
  const double mx = h[0] / N, my = h[2] / N;
  out[0] = my;
  out[1] = std::sqrt(std::max(0.0, (h[3] - N * my * my) / (N - 1.0)) / N);
  out[2] = mx;
  out[3] = std::sqrt(std::max(0.0, (h[1] - N * mx * mx) / (N - 1.0)) / N);
  return PC_OK;
}

pc_status pc_cv_beta(const pc_model *m, const pc_contract *k, const pc_cv_desc *c, const float *d_tables,
                     uint64_t n_paths, uint64_t seed, double *beta) {
  if (!beta) return fail(PC_EINVAL, "null output");
  if (n_paths < 16) return fail(PC_EINVAL, "n_paths must be >= 16");
  if (!m) return fail(PC_EINVAL, "null model");
  pc_ctx *ctx = m->ctx;
  pc_status s = cv_launch(m, k, c, d_tables, n_paths, seed, ctx->d_gout, nullptr, true);
  if (s != PC_OK) return s;
  double h[8];
  s = cv_sums(ctx, 8, h);
  if (s != PC_OK) return s;
  // moments: X, M, M2, XM, XM2, MM, M2M2, MM2
  const double N = double(n_paths);
  const double mx = h[0] / N, mm = h[1] / N, m2 = h[2] / N;
  const double cxm = h[3] / N - mx * mm, cxm2 = h[4] / N - mx * m2;
  const double vm = h[5] / N - mm * mm, vm2 = h[6] / N - m2 * m2, cmm2 = h[7] / N - mm * m2;
  if (c->use_gamma) {
    const double det = vm * vm2 - cmm2 * cmm2;
    if (det > 0.0) {
      beta[0] = (cxm * vm2 - cxm2 * cmm2) / det;
      beta[1] = (cxm2 * vm - cxm * cmm2) / det;
      return PC_OK;
    }
  }
  beta[0] = vm > 0.0 ? cxm / vm : 0.0;
  beta[1] = 0.0;
  return PC_OK;
}

pc_status pc_debug_cv_paths(const pc_model *m, const pc_contract *k, const pc_cv_desc *c, const float *d_tables,
                            uint64_t n_paths, uint64_t seed, float *d_xm) {
  if (!m || !d_xm) return fail(PC_EINVAL, "null argument");
  return cv_launch(m, k, c, d_tables, n_paths, seed, m->ctx->d_gout, d_xm, false);
}

}  // extern "C"
