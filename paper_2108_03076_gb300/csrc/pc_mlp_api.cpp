// pc_mlp_api.cpp -- pc_mlp_* entry points: parameter layout, buffers, the
// forward / backward / Adam launch sequences of pc_mlp.cu and the CUDA
// graph that replays one training step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "pc_handles.h"
#include "pc_mlp.h"

using namespace pc;

namespace {

constexpr int kPad = 64;
constexpr int kMaxLayers = 8;

int pad64(int x) { return (x + kPad - 1) / kPad * kPad; }

// splitmix64 (Steele, Lea & Flood, OOPSLA'14) for the initial weights.
uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct pc_mlp {
  pc_ctx *ctx = nullptr;
  int L = 0;
  std::vector<int> w, wp;           // real and padded widths [L + 1]
  std::vector<size_t> offW, offB;   // padded flat offsets
  size_t n_flat = 0, n_real = 0;
  size_t max_rows = 0;              // padded rows per call
  uint64_t steps = 0;
  bool tc_withhold = false;         // failure test of the tensor-core product's bounded waits
  void *mem = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *pb = nullptr;
  __nv_bfloat16 *X = nullptr;
  std::vector<__nv_bfloat16 *> H;   // hidden activations, layers 0..L-2
  __nv_bfloat16 *dZ[2] = {nullptr, nullptr};
  float *Y = nullptr, *T = nullptr, *wts = nullptr;
  float *part = nullptr, *colscr = nullptr, *loss_part = nullptr;
  size_t part_cap = 0;
  double *loss = nullptr;
  uint64_t *step = nullptr;
  // training graph and the arguments it was captured with
  cudaGraphExec_t exec = nullptr;
  const float *g_x = nullptr, *g_t = nullptr;
  size_t g_n = 0, g_batch = 0;
  float g_lr = 0.f;
  uint64_t g_seed = 0;
  std::vector<float> g_w;
  float *scratch = nullptr;         // caller scratch (mlp_scratch), grow-only
  size_t scratch_cap = 0;
  int32_t *dstatus = nullptr;       // device status of the tensor-core products
  int32_t gemm = PC_MLP_GEMM_AUTO;  // product kernel choice (pc_mlp_set_gemm)
  bool tc_ok = false;               // tcgen05 products available on this device
  std::map<uint64_t, TcMaps> tc_maps;  // operand descriptors by (product kind, layer, rows)
  float *h_pin = nullptr;             // pinned [8]: read-back of captured table builds
  std::vector<std::pair<std::vector<uint8_t>, cudaGraphExec_t>> graphs;  // captured table builds
};

namespace pc {
void mlp_drop_graphs(pc_mlp *N);

float *mlp_scratch(pc_mlp *N, size_t floats) {
  if (floats <= N->scratch_cap) return N->scratch;
  if (wait_stream(N->ctx) != PC_OK) return nullptr;
  mlp_drop_graphs(N);
  if (N->scratch) cudaFree(N->scratch);
  N->scratch = nullptr;
  N->scratch_cap = 0;
  if (cudaMalloc(&N->scratch, floats * sizeof(float)) != cudaSuccess) return nullptr;
  N->scratch_cap = floats;
  return N->scratch;
}

pc_status mlp_status(pc_mlp *N) {
  int32_t st = 0;
  CU(cudaMemcpyAsync(&st, N->dstatus, sizeof(st), cudaMemcpyDeviceToHost, N->ctx->stream), "status copy");
  pc_status r = wait_stream(N->ctx);
  if (r != PC_OK) return r;
  if (st == 0) return PC_OK;
  CU(cudaMemsetAsync(N->dstatus, 0, sizeof(st), N->ctx->stream), "status reset");
  wait_stream(N->ctx);
  return fail(PC_ETIMEOUT, "tensor-core product: a bounded wait expired");
}

}  // namespace pc

namespace {

struct Carve {
  char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T *r = reinterpret_cast<T *>(base + off);
    off += count * sizeof(T);
    return r;
  }
};

// Splits of the weight-gradient product over `rows`: enough blocks to cover
// the GPU, k ranges in whole 32-row steps.
int grad_splits(const pc_mlp *N, int M, int Nn, size_t rows, int &k_split) {
  const int tiles = (M / 64) * (Nn / 64);
  int want = std::max(1, (2 * N->ctx->sm_count + tiles - 1) / tiles);
  const int steps32 = int(rows / 32);
  want = std::min(want, steps32);
  k_split = ((steps32 + want - 1) / want) * 32;
  return int((rows + k_split - 1) / k_split);
}

// The same for the tensor-core weight gradient: 128 x (64 or 128) output
// tiles, k ranges in whole 64-row chunks.
int tc_grad_splits(const pc_mlp *N, int M, int Nn, size_t rows, int &k_split) {
  const int tiles = ((M + 127) / 128) * (Nn == 64 ? 1 : Nn / 128);
  int want = std::max(1, (2 * N->ctx->sm_count + tiles - 1) / tiles);
  const int steps64 = int(rows / 64);
  want = std::max(1, std::min(want, steps64));
  k_split = ((steps64 + want - 1) / want) * 64;
  return int((rows + k_split - 1) / k_split);
}

// Parameter offsets and the device buffers for `rows` padded rows, carved
// from N->mem; with N->mem null only the size is computed.
size_t layout(pc_mlp *N, size_t rows) {
  size_t flat = 0;
  N->offW.assign(N->L, 0);
  N->offB.assign(N->L, 0);
  for (int l = 0; l < N->L; ++l) {
    N->offW[l] = flat;
    flat += size_t(N->wp[l + 1]) * N->wp[l];
    N->offB[l] = flat;
    flat += size_t(N->wp[l + 1]);
  }
  N->n_flat = flat;
  int widest = 0;
  for (int x : N->wp) widest = std::max(widest, x);
  size_t part = 0;  // split-k partials: the largest layer at its split count
  for (int l = 0; l < N->L; ++l) {
    int ks = 0;
    const int sp = grad_splits(N, N->wp[l + 1], N->wp[l], rows, ks);
    part = std::max(part, size_t(sp) * N->wp[l + 1] * N->wp[l]);
    if (rows % 64 == 0) {
      const int tsp = tc_grad_splits(N, N->wp[l + 1], N->wp[l], rows, ks);
      part = std::max(part, size_t(tsp) * N->wp[l + 1] * N->wp[l]);
    }
  }
  N->part_cap = part;
  const size_t chunks = (rows + 255) / 256;
  Carve c{static_cast<char *>(N->mem)};
  N->p = c.take<float>(flat);
  N->g = c.take<float>(flat);
  N->m = c.take<float>(flat);
  N->v = c.take<float>(flat);
  N->pb = c.take<__nv_bfloat16>(flat);
  N->X = c.take<__nv_bfloat16>(rows * N->wp[0]);
  N->H.assign(std::max(0, N->L - 1), nullptr);
  for (int l = 0; l + 1 < N->L; ++l) N->H[l] = c.take<__nv_bfloat16>(rows * N->wp[l + 1]);
  N->dZ[0] = c.take<__nv_bfloat16>(rows * widest);
  N->dZ[1] = c.take<__nv_bfloat16>(rows * widest);
  N->Y = c.take<float>(rows * N->wp[N->L]);
  N->T = c.take<float>(rows * N->wp[N->L]);
  N->wts = c.take<float>(kPad);
  N->part = c.take<float>(part);
  N->colscr = c.take<float>(chunks * widest);
  N->loss_part = c.take<float>(512);
  N->loss = c.take<double>(1);
  N->step = c.take<uint64_t>(1);
  N->dstatus = c.take<int32_t>(1);
  return c.off;
}

GemmArgs gemm0() {
  GemmArgs a;
  std::memset(&a, 0, sizeof(a));
  return a;
}

// One product: on the tensor cores when they serve this shape (operand
// descriptors cached by kind, layer and rows), else the warp-level kernel.
// A weight gradient is split over k differently on each path (splits and
// a.k_split on the warp-level kernel, tc_splits and tc_k_split on the tensor
// cores); *used receives the split count of the path taken.
cudaError_t product(pc_mlp *N, GemmKind kind, int epi, int layer, size_t rows, GemmArgs a, int splits,
                    int tc_k_split, int tc_splits, cudaStream_t s, int *used = nullptr) {
  if (used) *used = splits;
  if (N->tc_ok && N->gemm == PC_MLP_GEMM_AUTO) {
    GemmArgs t = a;
    if (kind == kGemmWeightGrad) t.k_split = tc_k_split;
    if (gemm_tc_supported(kind, t)) {
      const uint64_t key = (uint64_t(kind) << 56) | (uint64_t(layer) << 40) | uint64_t(rows);
      auto it = N->tc_maps.find(key);
      if (it == N->tc_maps.end()) {
        TcMaps m;
        if (make_tc_maps(kind, t, m)) it = N->tc_maps.emplace(key, m).first;
      }
      if (it != N->tc_maps.end()) {
        const int sp = kind == kGemmWeightGrad ? tc_splits : 1;
        if (used) *used = sp;
        return launch_gemm_tc(kind, epi, t, it->second, sp, N->dstatus, s, N->tc_withhold);
      }
    }
  }
  return launch_gemm(kind, epi, a, splits, s);
}

// Forward over `rows` padded rows already in X.
cudaError_t forward(pc_mlp *N, size_t rows, cudaStream_t s) {
  for (int l = 0; l < N->L; ++l) {
    GemmArgs a = gemm0();
    a.A = l == 0 ? N->X : N->H[l - 1];
    a.lda = N->wp[l];
    a.B = N->pb + N->offW[l];
    a.ldb = N->wp[l];
    a.M = int(rows);
    a.N = N->wp[l + 1];
    a.K = N->wp[l];
    a.k_split = a.K;
    a.bias = N->p + N->offB[l];
    const bool last = l == N->L - 1;
    if (last) {
      a.Cf = N->Y;
    } else {
      a.Cb = N->H[l];
    }
    a.ldc = N->wp[l + 1];
    const int epi = last ? kEpiBias : kEpiBiasSoftplus;
    cudaError_t e = product(N, kGemmForward, epi, l, rows, a, 1, 0, 1, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Loss on the first n of `rows` rows (targets in T), gradients into g.
cudaError_t backward(pc_mlp *N, size_t n, size_t rows, cudaStream_t s) {
  const int fout = N->w[N->L];
  const int lb = loss_blocks(rows);
  cudaError_t e = launch_loss(N->Y, N->wp[N->L], N->T, N->wts, n, fout, rows, N->dZ[0], N->wp[N->L],
                              N->loss_part, lb, s);
  if (e != cudaSuccess) return e;
  int cur = 0;
  for (int l = N->L - 1; l >= 0; --l) {
    const __nv_bfloat16 *in = l == 0 ? N->X : N->H[l - 1];
    const int out_w = N->wp[l + 1], in_w = N->wp[l];
    // dW_l = dZ^T in
    GemmArgs a = gemm0();
    a.A = N->dZ[cur];
    a.lda = out_w;
    a.B = in;
    a.ldb = in_w;
    a.M = out_w;
    a.N = in_w;
    a.K = int(rows);
    int splits = grad_splits(N, out_w, in_w, rows, a.k_split);
    int tc_ks = 0;
    const int tc_splits = rows % 64 == 0 ? tc_grad_splits(N, out_w, in_w, rows, tc_ks) : 0;
    a.Cf = N->part;
    a.ldc = in_w;
    e = product(N, kGemmWeightGrad, kEpiPartial, l, rows, a, splits, tc_ks, tc_splits, s, &splits);
    if (e != cudaSuccess) return e;
    const size_t cnt = size_t(out_w) * in_w;
    e = launch_split_sum(N->part, splits, cnt, cnt, N->g + N->offW[l], s);
    if (e != cudaSuccess) return e;
    e = launch_colsum(N->dZ[cur], rows, out_w, out_w, N->colscr, N->g + N->offB[l], s);
    if (e != cudaSuccess) return e;
    if (l > 0) {
      // dZ_{l-1} = (dZ_l W_l) * softplus'(z_{l-1})
      GemmArgs b = gemm0();
      b.A = N->dZ[cur];
      b.lda = out_w;
      b.B = N->pb + N->offW[l];
      b.ldb = in_w;
      b.M = int(rows);
      b.N = in_w;
      b.K = out_w;
      b.k_split = out_w;
      b.aux = N->H[l - 1];
      b.ldaux = in_w;
      b.Cb = N->dZ[cur ^ 1];
      b.ldc = in_w;
      e = product(N, kGemmDataGrad, kEpiDSoftplus, l, rows, b, 1, 0, 1, s);
      if (e != cudaSuccess) return e;
      cur ^= 1;
    }
  }
  return cudaSuccess;
}

size_t rows_for(size_t n) { return (n + 63) / 64 * 64; }

pc_status upload_padded(pc_mlp *N, const float *host) {
  std::vector<float> flat(N->n_flat, 0.f);
  size_t k = 0;
  for (int l = 0; l < N->L; ++l) {
    for (int o = 0; o < N->w[l + 1]; ++o)
      for (int i = 0; i < N->w[l]; ++i) flat[N->offW[l] + size_t(o) * N->wp[l] + i] = host[k++];
    for (int o = 0; o < N->w[l + 1]; ++o) flat[N->offB[l] + o] = host[k++];
  }
  std::vector<__nv_bfloat16> fb(N->n_flat);
  for (size_t i = 0; i < N->n_flat; ++i) fb[i] = __float2bfloat16_rn(flat[i]);
  cudaStream_t s = N->ctx->stream;
  CU(cudaMemcpyAsync(N->p, flat.data(), N->n_flat * 4, cudaMemcpyHostToDevice, s), "params");
  CU(cudaMemcpyAsync(N->pb, fb.data(), N->n_flat * 2, cudaMemcpyHostToDevice, s), "params");
  CU(cudaMemsetAsync(N->m, 0, N->n_flat * 4, s), "moments");
  CU(cudaMemsetAsync(N->v, 0, N->n_flat * 4, s), "moments");
  CU(cudaMemsetAsync(N->step, 0, 8, s), "step");
  N->steps = 0;
  return wait_stream(N->ctx);
}

// Device gather of a padded flat array into the unpadded layout.
pc_status copy_unpadded(pc_mlp *N, const float *src, float *dst, cudaMemcpyKind kind) {
  cudaStream_t s = N->ctx->stream;
  size_t k = 0;
  for (int l = 0; l < N->L; ++l) {
    const size_t o = N->w[l + 1], i = N->w[l];
    CU(cudaMemcpy2DAsync(dst + k, i * 4, src + N->offW[l], size_t(N->wp[l]) * 4, i * 4, o, kind, s),
       "parameter copy");
    k += o * i;
    CU(cudaMemcpyAsync(dst + k, src + N->offB[l], o * 4, kind, s), "parameter copy");
    k += o;
  }
  return PC_OK;
}

pc_status set_weights(pc_mlp *N, const float *w) {
  float h[kPad] = {0};
  for (int j = 0; j < N->w[N->L]; ++j) h[j] = w[j];
  CU(cudaMemcpyAsync(N->wts, h, sizeof(h), cudaMemcpyHostToDevice, N->ctx->stream), "loss weights");
  return PC_OK;
}

}  // namespace

namespace pc {

void mlp_drop_graphs(pc_mlp *N) {
  for (auto &g : N->graphs)
    if (g.second) cudaGraphExecDestroy(g.second);
  N->graphs.clear();
}

cudaGraphExec_t *mlp_graph(pc_mlp *N, const std::vector<uint8_t> &key) {
  for (auto &g : N->graphs)
    if (g.first == key) return &g.second;
  if (N->graphs.size() >= 16) mlp_drop_graphs(N);
  N->graphs.emplace_back(key, nullptr);
  return &N->graphs.back().second;
}

float *mlp_pinned(pc_mlp *N) { return N->h_pin; }
int32_t *mlp_status_word(pc_mlp *N) { return N->dstatus; }

// The fused table build's network description (cv_tables_tc): false when
// the products do not run on tcgen05 or the network's shape is outside the
// kernel's (then the caller builds the tables with the layer products).
bool mlp_cv_tables_tc(pc_mlp *N, size_t rows, float *tables, float *delta0, CvTablesTc &t) {
  if (!N->tc_ok || N->gemm != PC_MLP_GEMM_AUTO || !cv_tables_tc_shape(N->L, N->wp.data())) return false;
  std::memset(&t, 0, sizeof(t));
  t.L = N->L;
  for (int l = 0; l <= N->L; ++l) t.wp[l] = N->wp[l];
  for (int l = 0; l < N->L; ++l) {
    // the weight map of layer l, encoded once per network
    const uint64_t key = (uint64_t(7) << 56) | uint64_t(l);
    auto it = N->tc_maps.find(key);
    if (it == N->tc_maps.end()) {
      TcMaps mm;
      if (!make_weight_map(mm.b, N->pb + N->offW[l], N->wp[l + 1], N->wp[l])) return false;
      it = N->tc_maps.emplace(key, mm).first;
    }
    t.w[l] = it->second.b;
    t.bias[l] = N->p + N->offB[l];
  }
  t.rows = rows;
  t.tables = tables;
  t.delta0 = delta0;
  t.status = N->dstatus;
  t.withhold = N->tc_withhold ? 1 : 0;
  return true;
}

pc_status mlp_forward_on(pc_mlp *N, const float *d_x, size_t n, float *d_y, cudaStream_t s) {
  for (size_t b0 = 0; b0 < n; b0 += N->max_rows) {
    const size_t nb = std::min(N->max_rows, n - b0), rows = rows_for(nb);
    CU(launch_to_bf16(d_x + b0 * N->w[0], nb, N->w[0], N->X, rows, N->wp[0], s), "input");
    CU(forward(N, rows, s), "forward");
    CU(launch_unpad(N->Y, N->wp[N->L], nb, N->w[N->L], d_y + b0 * N->w[N->L], s), "output");
  }
  return PC_OK;
}
}  // namespace pc

extern "C" {

pc_status pc_mlp_create(pc_ctx *c, const int32_t *widths, int32_t n_widths, uint64_t max_batch,
                        uint64_t seed, pc_mlp **out) {
  if (!c || !widths || !out) return fail(PC_EINVAL, "null argument");
  if (n_widths < 2 || n_widths > kMaxLayers + 1) return fail(PC_EINVAL, "n_widths must be 2..9");
  if (max_batch < 1 || max_batch > (uint64_t(1) << 24)) return fail(PC_EINVAL, "max_batch must be 1..2^24");
  for (int i = 0; i < n_widths; ++i) {
    const bool edge = i == 0 || i == n_widths - 1;
    if (widths[i] < 1 || (edge && widths[i] > kPad) || (!edge && (widths[i] % kPad || widths[i] > 1024)))
      return fail(PC_EINVAL, "widths: input/output 1..64, hidden multiples of 64 up to 1024");
  }
  pc_mlp *N = new (std::nothrow) pc_mlp;
  if (!N) return fail(PC_ENOMEM, "network");
  N->ctx = c;
  N->L = n_widths - 1;
  N->w.assign(widths, widths + n_widths);
  N->wp.resize(n_widths);
  for (int i = 0; i < n_widths; ++i) N->wp[i] = pad64(widths[i]);
  N->max_rows = rows_for(max_batch);
  N->n_real = 0;
  for (int l = 0; l < N->L; ++l) N->n_real += size_t(N->w[l + 1]) * (N->w[l] + 1);
  const size_t bytes = layout(N, N->max_rows);
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess) e = cudaMalloc(&N->mem, bytes);
  if (e != cudaSuccess) {
    delete N;
    return cuda_fail(e, "network memory");
  }
  layout(N, N->max_rows);
  std::vector<float> init(N->n_real);
  uint64_t st = seed;
  size_t k = 0;
  for (int l = 0; l < N->L; ++l) {
    const float a = 1.0f / std::sqrt(float(N->w[l]));
    const size_t cnt = size_t(N->w[l + 1]) * (N->w[l] + 1);
    for (size_t i = 0; i < cnt; ++i) {
      const double u = double(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      init[k++] = float((2.0 * u - 1.0) * a);
    }
  }
  cudaMemsetAsync(N->mem, 0, bytes, c->stream);
  N->tc_ok = gemm_tc_init() == cudaSuccess;
  cudaGetLastError();
  if (cudaHostAlloc(reinterpret_cast<void **>(&N->h_pin), 8 * sizeof(float), 0) != cudaSuccess) {
    N->h_pin = nullptr;
    cudaGetLastError();
  }
  pc_status s = upload_padded(N, init.data());
  if (s != PC_OK) {
    cudaFree(N->mem);
    delete N;
    return s;
  }
  *out = N;
  return PC_OK;
}

pc_status pc_mlp_destroy(pc_mlp *N) {
  if (!N) return fail(PC_EINVAL, "null network");
  cudaSetDevice(N->ctx->device);
  wait_stream(N->ctx);
  if (N->exec) cudaGraphExecDestroy(N->exec);
  mlp_drop_graphs(N);
  if (N->h_pin) cudaFreeHost(N->h_pin);
  if (N->mem) cudaFree(N->mem);
  if (N->scratch) cudaFree(N->scratch);
  delete N;
  return PC_OK;
}

pc_status pc_mlp_query(const pc_mlp *N, pc_mlp_info *info) {
  if (!N || !info) return fail(PC_EINVAL, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->n_layers = N->L;
  for (int i = 0; i <= N->L; ++i) info->widths[i] = N->w[i];
  info->n_params = N->n_real;
  info->max_batch = N->max_rows;
  info->steps = N->steps;
  return PC_OK;
}

pc_status pc_mlp_set_params(pc_mlp *N, const float *params, size_t n) {
  if (!N || !params) return fail(PC_EINVAL, "null argument");
  if (n != N->n_real) return fail(PC_EINVAL, "parameter count mismatch");
  CU(cudaSetDevice(N->ctx->device), "cudaSetDevice");
  return upload_padded(N, params);
}

pc_status pc_mlp_get_params(const pc_mlp *N, float *params, size_t n) {
  if (!N || !params) return fail(PC_EINVAL, "null argument");
  if (n != N->n_real) return fail(PC_EINVAL, "parameter count mismatch");
  auto *M = const_cast<pc_mlp *>(N);
  CU(cudaSetDevice(N->ctx->device), "cudaSetDevice");
  pc_status s = copy_unpadded(M, N->p, params, cudaMemcpyDeviceToHost);
  if (s != PC_OK) return s;
  return wait_stream(N->ctx);
}

pc_status pc_mlp_forward(pc_mlp *N, const float *d_x, size_t n, float *d_y) {
  if (!N || (n && (!d_x || !d_y))) return fail(PC_EINVAL, "null argument");
  CU(cudaSetDevice(N->ctx->device), "cudaSetDevice");
  return mlp_forward_on(N, d_x, n, d_y, N->ctx->stream);
}

pc_status pc_mlp_gradients(pc_mlp *N, const float *d_x, const float *d_t, const float *w, size_t n,
                           float *d_grads, double *out_loss) {
  if (!N || !d_x || !d_t || !w || !out_loss) return fail(PC_EINVAL, "null argument");
  if (n < 1 || n > N->max_rows) return fail(PC_EINVAL, "n must be 1..max_batch");
  cudaStream_t s = N->ctx->stream;
  CU(cudaSetDevice(N->ctx->device), "cudaSetDevice");
  const size_t rows = rows_for(n);
  pc_status st = set_weights(N, w);
  if (st != PC_OK) return st;
  CU(launch_to_bf16(d_x, n, N->w[0], N->X, rows, N->wp[0], s), "input");
  CU(cudaMemcpyAsync(N->T, d_t, n * N->w[N->L] * sizeof(float), cudaMemcpyDeviceToDevice, s), "targets");
  CU(forward(N, rows, s), "forward");
  CU(backward(N, n, rows, s), "backward");
  CU(launch_loss_total(N->loss_part, loss_blocks(rows), N->loss, nullptr, s), "loss");
  if (d_grads) {
    st = copy_unpadded(N, N->g, d_grads, cudaMemcpyDeviceToDevice);
    if (st != PC_OK) return st;
  }
  CU(cudaMemcpyAsync(out_loss, N->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "loss copy");
  return mlp_status(N);
}

pc_status pc_mlp_train(pc_mlp *N, const float *d_x, const float *d_t, size_t n_data, const float *w,
                       size_t batch, int32_t steps, float lr, uint64_t seed, double *out_loss) {
  if (!N || !d_x || !d_t || !w || !out_loss) return fail(PC_EINVAL, "null argument");
  if (n_data < 1 || batch < 1 || batch > N->max_rows) return fail(PC_EINVAL, "n_data >= 1, batch 1..max_batch");
  if (steps < 0) return fail(PC_EINVAL, "steps must be >= 0");
  if (!(lr > 0.f)) return fail(PC_EINVAL, "lr must be > 0");
  pc_ctx *c = N->ctx;
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  std::vector<float> wv(w, w + N->w[N->L]);
  const bool same = N->exec && N->g_x == d_x && N->g_t == d_t && N->g_n == n_data && N->g_batch == batch &&
                    N->g_lr == lr && N->g_seed == seed && N->g_w == wv;
  if (!same) {
    if (N->exec) cudaGraphExecDestroy(N->exec);
    N->exec = nullptr;
    pc_status st = set_weights(N, w);
    if (st != PC_OK) return st;
    st = wait_stream(c);
    if (st != PC_OK) return st;
    cudaStream_t cap = nullptr;
    CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    const size_t rows = rows_for(batch);
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      if (rows > batch) e = cudaMemsetAsync(N->X, 0, rows * N->wp[0] * sizeof(__nv_bfloat16), cap);
      if (e == cudaSuccess)
        e = launch_gather(d_x, d_t, n_data, N->w[0], N->w[N->L], N->step, uint32_t(seed), uint32_t(seed >> 32),
                          batch, N->X, N->wp[0], N->T, cap);
      if (e == cudaSuccess) e = forward(N, rows, cap);
      if (e == cudaSuccess) e = backward(N, batch, rows, cap);
      if (e == cudaSuccess)
        e = launch_adam(N->p, N->g, N->m, N->v, N->pb, N->n_flat, N->step, lr, 0.9f, 0.999f, 1e-8f, cap);
      if (e == cudaSuccess) e = launch_loss_total(N->loss_part, loss_blocks(rows), N->loss, N->step, cap);
      cudaGraph_t graph = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&N->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      N->exec = nullptr;
      return cuda_fail(e, "training graph");
    }
    N->g_x = d_x;
    N->g_t = d_t;
    N->g_n = n_data;
    N->g_batch = batch;
    N->g_lr = lr;
    N->g_seed = seed;
    N->g_w = wv;
  }
  for (int32_t i = 0; i < steps; ++i) CU(cudaGraphLaunch(N->exec, c->stream), "training step");
  CU(cudaMemcpyAsync(out_loss, N->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "loss copy");
  pc_status st = mlp_status(N);
  if (st != PC_OK) return st;
  N->steps += uint64_t(steps);
  return PC_OK;
}

pc_status pc_debug_mlp_withhold_tma(pc_mlp *N, int32_t on) {
  if (!N) return fail(PC_EINVAL, "null network");
  wait_stream(N->ctx);
  mlp_drop_graphs(N);
  if (N->exec) cudaGraphExecDestroy(N->exec);
  N->exec = nullptr;
  N->tc_withhold = on != 0;
  return PC_OK;
}

pc_status pc_mlp_set_gemm(pc_mlp *N, int32_t kind) {
  if (!N) return fail(PC_EINVAL, "null network");
  if (kind != PC_MLP_GEMM_AUTO && kind != PC_MLP_GEMM_MMA_SYNC) return fail(PC_EINVAL, "unknown product kind");
  if (kind != N->gemm) {
    wait_stream(N->ctx);
    if (N->exec) cudaGraphExecDestroy(N->exec);  // the training step is captured again
    N->exec = nullptr;
    mlp_drop_graphs(N);
    N->gemm = kind;
  }
  return PC_OK;
}

pc_status pc_mlp_gemm_info(const pc_mlp *N, int32_t *tensor_cores) {
  if (!N || !tensor_cores) return fail(PC_EINVAL, "null argument");
  *tensor_cores = N->tc_ok && N->gemm == PC_MLP_GEMM_AUTO ? 1 : 0;
  return PC_OK;
}

}  // extern "C"
