// pc_batch.cpp -- portfolio pricing plans (pc_batch_*) and pc_price_batch.
//
// A plan validates every (model, contract, n_paths) exactly as pc_price does,
// keeps one PriceArgs per contract in device memory, groups the contracts by
// underlying count and per-path shared-memory footprint, cuts each
// contract's tiles into work units and captures the group launches (one
// persistent batch_kernel per group, all groups as parallel graph branches
// after one memset of the reduction scratch) into a CUDA graph.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "pc_handles.h"
#include "pc_internal.h"

using namespace pc;

namespace {

constexpr int kMaxGroups = 64;
constexpr size_t kCounterBytes = kMaxGroups * sizeof(unsigned long long);

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Group {
  int d = 0;
  int words = 0;            // largest per-path shared words of its contracts
  size_t slot = 0;          // largest per-warp slot (arguments + program + pool)
  int block = 0;
  size_t smem = 0;
  int grid = 0;
  uint32_t u0 = 0, n_units = 0;
  std::vector<uint32_t> items;
};

}  // namespace

struct pc_batch {
  pc_ctx *ctx = nullptr;
  size_t n = 0;
  std::vector<PriceArgs> items;     // device pointers filled in
  std::vector<int> d, words;
  std::vector<double> tile_cost;    // estimated cost of one 64-path tile
  std::vector<uint64_t> n_paths;
  uint64_t total_tiles = 0;
  double total_cost = 0.0;
  std::vector<Group> groups;
  // device memory: one allocation
  void *d_mem = nullptr;
  PriceArgs *d_items = nullptr;
  BatchUnit *d_units = nullptr;
  unsigned char *d_zero = nullptr;  // group counters, then per-contract control blocks
  size_t zero_bytes = 0;
  double *d_out = nullptr;          // [4n]: sum x, sum x^2, n, -
  // graph
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> aux;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t exec = nullptr;
  pc_batch_config cfg{128, 128};
  uint64_t n_units = 0;
  double paths_per_thread = 0.0;
  bool tuned = false;
  bool single = false;              // one launch of batch_kernel_any for every contract
  double last_ms = 0.0;
  // contracts priced by their run-time specialised kernel, each its own
  // branch of the graph (the costliest, with the context's pc_set_jit)
  struct JitItem {
    uint32_t item = 0;
    cudaKernel_t kern = nullptr;
    int grid = 0, block = 0;
    size_t smem = 0;
    PriceArgs args{};
  };
  std::vector<JitItem> jit;
  std::vector<char> is_jit;
};

namespace {

// Estimated cost of one tile: generation of every model date for every
// underlying (normals, bridge, correlation, exponentials) plus one pass
// over the program; only the order of units and their lengths depend on it.
double estimate_tile_cost(const PriceArgs &a, int d) {
  return double(a.m.n) * (4.0 * d + 2.0) + double(a.n_insn) + 8.0;
}

int words_class(int words) {
  int c = 0;
  while ((16 << c) < words) ++c;
  return c;
}

// Contracts grouped by (underlying count, power-of-two class of per-path
// shared words): one persistent launch per group, sized for its largest
// footprint.  In single-launch mode every contract is in one group (d = 0:
// batch_kernel_any, sized for the largest footprint of all).
void build_groups(pc_batch *B) {
  std::map<std::pair<int, int>, uint32_t> index;
  B->groups.clear();
  for (size_t i = 0; i < B->n; ++i) {
    if (!B->single && !B->is_jit.empty() && B->is_jit[i]) continue;  // its own specialised launch
    const auto key = B->single ? std::make_pair(0, 0) : std::make_pair(B->d[i], words_class(B->words[i]));
    auto it = index.find(key);
    if (it == index.end()) {
      it = index.emplace(key, uint32_t(B->groups.size())).first;
      Group g;
      g.d = B->single ? 0 : B->d[i];
      B->groups.push_back(g);
    }
    Group &g = B->groups[it->second];
    g.items.push_back(uint32_t(i));
    g.words = std::max(g.words, B->words[i]);
    g.slot = std::max(g.slot, batch_slot_bytes(size_t(B->items[i].n_insn), size_t(B->items[i].n_pool)));
  }
}

void destroy_graph(pc_batch *B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  B->exec = nullptr;
}

// Block size (<= the preferred one) with the most resident warps per SM for
// a group's footprint; 0 if none fits.
int group_block(const Group &g, int preferred, int max_smem, size_t &smem, int &bpsm) {
  int best = 0, best_warps = 0;
  for (int b = kBlock; b >= 32; b /= 2) {
    if (b > preferred) continue;
    const size_t sm = batch_smem_bytes(g.slot, g.words, b);
    if (sm + kStaticSmemReserve > size_t(max_smem)) continue;
    const int nb = batch_blocks_per_sm(g.d, b, sm);
    if (nb * (b / 32) > best_warps) {
      best = b;
      best_warps = nb * (b / 32);
      smem = sm;
      bpsm = nb;
    }
  }
  return best;
}

// Work units under a launch shape, the group launch shapes, the unit upload
// and the graph.
pc_status configure(pc_batch *B, const pc_batch_config &cfg) {
  pc_ctx *c = B->ctx;
  if (cfg.block != 32 && cfg.block != 64 && cfg.block != 128)
    return fail(PC_EINVAL, "batch block must be 32, 64 or 128");
  if (cfg.unit_split < 1 || cfg.unit_split > (1 << 16))
    return fail(PC_EINVAL, "batch unit_split must be 1..65536");
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  // the previous graph may still be running: units are rewritten below
  pc_status s = wait_stream(c);
  if (s != PC_OK) return s;
  destroy_graph(B);
  const double warps = double(c->sm_count) * 16.0;
  const double target = B->total_cost / warps / double(cfg.unit_split);
  std::vector<BatchUnit> units;
  units.reserve(size_t(B->total_tiles));
  double thread_paths = 0.0;
  for (Group &g : B->groups) {
    g.u0 = uint32_t(units.size());
    std::vector<std::pair<double, BatchUnit>> gu;
    for (uint32_t i : g.items) {
      const uint64_t nt = B->items[i].n_tiles;
      uint64_t per = uint64_t(std::floor(target / B->tile_cost[i]));
      per = std::min<uint64_t>(std::max<uint64_t>(per, 1), nt);
      per = std::min<uint64_t>(per, 1u << 20);
      for (uint64_t t0 = 0; t0 < nt; t0 += per) {
        BatchUnit u;
        u.item = i;
        u.tile0 = t0;
        u.n_tiles = uint32_t(std::min<uint64_t>(per, nt - t0));
        gu.emplace_back(double(u.n_tiles) * B->tile_cost[i], u);
        thread_paths += 2.0 * u.n_tiles;
      }
    }
    // costliest first (longest-processing-time order); ties by contract, tile
    std::stable_sort(gu.begin(), gu.end(), [](const auto &x, const auto &y) {
      if (x.first != y.first) return x.first > y.first;
      if (x.second.item != y.second.item) return x.second.item < y.second.item;
      return x.second.tile0 < y.second.tile0;
    });
    for (const auto &p : gu) units.push_back(p.second);
    g.n_units = uint32_t(units.size() - g.u0);
  }
  B->n_units = units.size();
  B->paths_per_thread = units.empty() ? 0.0 : thread_paths / double(units.size());
  // group shapes
  for (Group &g : B->groups) {
    int bpsm = 0;
    g.block = group_block(g, cfg.block, c->max_smem, g.smem, bpsm);
    if (!g.block)
      return fail(PC_ELIMIT, "per-path state of a batch group (" + std::to_string(g.words) +
                                 " shared words per thread) exceeds shared memory");
    const uint64_t wpb = uint64_t(g.block / 32);
    const uint64_t need = (uint64_t(g.n_units) + wpb - 1) / wpb;
    g.grid = int(std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(c->sm_count) * bpsm, need)));
  }
  // leave each kernel's dynamic shared-memory limit at its largest group
  for (const Group &g : B->groups) {
    size_t mx = 0;
    for (const Group &h : B->groups)
      if (h.d == g.d) mx = std::max(mx, h.smem);
    if (batch_blocks_per_sm(g.d, 32, mx) < 1)
      return fail(PC_ELIMIT, "batch kernel cannot be resident");
  }
  if (!units.empty())
    CU(cudaMemcpy(B->d_units, units.data(), units.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice),
       "unit upload");
  B->cfg = cfg;
  return PC_OK;
}

// With the context's pc_set_jit: the costliest contracts (by estimated tile
// cost x tiles, until kBatchJitShare of the portfolio's cost or kBatchJitMax
// contracts; at least kBatchJitMinTiles tiles each) priced by their
// run-time specialised kernel on their own graph branch instead of the
// interpreting group kernels -- the same per-tile work and reduction, so
// the same bits.  Their arguments are the plan's, with the specialised
// kernel's layout.
constexpr size_t kBatchJitMax = 160;
constexpr double kBatchJitShare = 0.8;
constexpr uint64_t kBatchJitMinTiles = 64;

pc_status choose_jit(pc_batch *B, const pc_model *const *models, const pc_contract *const *contracts,
                     const uint64_t *n_paths, uint64_t seed) {
  pc_ctx *c = B->ctx;
  B->jit.clear();
  B->is_jit.assign(B->n, 0);
  if (!c->jit) return PC_OK;
  std::vector<uint32_t> order(B->n);
  for (size_t i = 0; i < B->n; ++i) order[i] = uint32_t(i);
  auto cost = [&](uint32_t i) { return double(B->items[i].n_tiles) * B->tile_cost[i]; };
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return cost(x) > cost(y); });
  // the candidates and their kernels' variants, compiled together
  struct Cand {
    uint32_t i;
    Launch L;
    int wk;
    size_t smem;
    int min_blocks;
  };
  std::vector<Cand> cand;
  std::vector<JitRequest> reqs;
  double est = 0.0;
  for (uint32_t i : order) {
    if (cand.size() >= kBatchJitMax || est >= kBatchJitShare * B->total_cost) break;
    if (B->items[i].n_tiles < kBatchJitMinTiles || !jit_eligible(contracts[i])) continue;
    Cand cd;
    cd.i = i;
    pc_status s = prepare(models[i], contracts[i], n_paths[i], 0, seed, i, cd.L);
    if (s != PC_OK) return s;
    cd.wk = jit_window_kind(c, cd.L);
    if (cd.wk & kJitHbm) continue;
    cd.smem = jit_layout(c, contracts[i], cd.L, cd.wk);
    cd.min_blocks = jit_min_blocks(c, cd.smem, cd.L.block);
    reqs.push_back({contracts[i], models[i]->H.d, kJitPrice | cd.wk, cd.L.block, cd.min_blocks});
    cand.push_back(cd);
    est += cost(i);
  }
  pc_status sc = jit_compile_many(c, reqs);
  if (sc != PC_OK) return sc;
  for (Cand &cd : cand) {
    const uint32_t i = cd.i;
    Launch &L = cd.L;
    const int wk = cd.wk;
    const size_t smem = cd.smem;
    cudaKernel_t jk = nullptr;
    pc_status s = jit_kernel(contracts[i], models[i]->H.d, kJitPrice | wk, L.block, jk, cd.min_blocks);
    if (s != PC_OK) return s;
    int nb = 0;
    CU(jit_occupancy(c, reinterpret_cast<const void *>(jk), L.block, smem, nb), "jit occupancy");
    if (nb < 1) continue;
    const uint64_t tiles = B->items[i].n_tiles;
    const uint64_t units = (wk & kJitPairs2) ? (tiles + 1) / 2 : tiles, wpb = uint64_t(L.block / 32);
    pc_batch::JitItem J;
    J.item = i;
    J.kern = jk;
    J.block = L.block;
    J.smem = smem;
    J.grid = int(std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(c->sm_count) * nb, (units + wpb - 1) / wpb)));
    J.args = B->items[i];
    J.args.lay = L.args.lay;
    B->jit.push_back(J);
    B->is_jit[i] = 1;
  }
  // a kernel shared by several contracts takes the largest of their
  // dynamic shared memory sizes
  for (const pc_batch::JitItem &J : B->jit) {
    size_t mx = 0;
    for (const pc_batch::JitItem &K : B->jit)
      if (K.kern == J.kern) mx = std::max(mx, K.smem);
    CU(cudaFuncSetAttribute(reinterpret_cast<const void *>(J.kern), cudaFuncAttributeMaxDynamicSharedMemorySize,
                            int(mx)), "specialised kernel shared memory");
  }
  return PC_OK;
}

// One specialised contract's launch (its PriceArgs by value).
cudaError_t launch_jit_item(const pc_batch::JitItem &J, cudaStream_t st) {
  PriceArgs a = J.args;
  void *args[] = {&a};
  return cudaLaunchKernel(reinterpret_cast<const void *>(J.kern), dim3(J.grid), dim3(J.block), args, J.smem, st);
}

// Capture: memset of the counters and control blocks, then every group's
// launch on its own branch, joined back into the capture stream.
pc_status capture(pc_batch *B) {
  pc_ctx *c = B->ctx;
  const size_t n_jit = B->single ? 0 : B->jit.size();
  while (B->aux.size() < B->groups.size() + n_jit) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
    B->aux.push_back(st);
    CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    B->joins.push_back(ev);
  }
  CU(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = cudaMemsetAsync(B->d_zero, 0, B->zero_bytes, B->cap);
  if (e == cudaSuccess) e = cudaEventRecord(B->fork, B->cap);
  for (size_t gi = 0; gi < B->groups.size() && e == cudaSuccess; ++gi) {
    const Group &g = B->groups[gi];
    if (g.n_units == 0) continue;
    BatchArgs a;
    a.items = B->d_items;
    a.units = B->d_units + g.u0;
    a.n_units = g.n_units;
    a.slot_bytes = uint32_t(g.slot);
    a.counter = reinterpret_cast<unsigned long long *>(B->d_zero) + gi;
    e = cudaStreamWaitEvent(B->aux[gi], B->fork, 0);
    if (e == cudaSuccess) e = launch_batch(a, g.d, g.grid, g.block, g.smem, B->aux[gi]);
    if (e == cudaSuccess) e = cudaEventRecord(B->joins[gi], B->aux[gi]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->cap, B->joins[gi], 0);
  }
  for (size_t j = 0; j < n_jit && e == cudaSuccess; ++j) {
    const size_t si = B->groups.size() + j;
    e = cudaStreamWaitEvent(B->aux[si], B->fork, 0);
    if (e == cudaSuccess) e = launch_jit_item(B->jit[j], B->aux[si]);
    if (e == cudaSuccess) e = cudaEventRecord(B->joins[si], B->aux[si]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->cap, B->joins[si], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(B->cap, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    B->exec = nullptr;
    return cuda_fail(e, "batch graph");
  }
  (void)c;
  return PC_OK;
}

pc_status launch(pc_batch *B) {
  CU(cudaSetDevice(B->ctx->device), "cudaSetDevice");
  CU(cudaGraphLaunch(B->exec, B->ctx->stream), "graph launch");
  return PC_OK;
}

// The plan's work without a graph (one-shot pricing): the same group
// launches as the captured replay, forked onto the context's cached
// streams and joined back into its stream.
pc_status launch_direct(pc_batch *B) {
  pc_ctx *c = B->ctx;
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  if (!c->batch_fork) CU(cudaEventCreateWithFlags(&c->batch_fork, cudaEventDisableTiming), "event");
  const size_t n_jit = B->single ? 0 : B->jit.size();
  while (c->batch_aux.size() < B->groups.size() + n_jit) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
    c->batch_aux.push_back(st);
    CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    c->batch_join.push_back(ev);
  }
  CU(cudaMemsetAsync(B->d_zero, 0, B->zero_bytes, c->stream), "counters");
  CU(cudaEventRecord(c->batch_fork, c->stream), "fork");
  for (size_t gi = 0; gi < B->groups.size(); ++gi) {
    const Group &g = B->groups[gi];
    if (g.n_units == 0) continue;
    BatchArgs a;
    a.items = B->d_items;
    a.units = B->d_units + g.u0;
    a.n_units = g.n_units;
    a.slot_bytes = uint32_t(g.slot);
    a.counter = reinterpret_cast<unsigned long long *>(B->d_zero) + gi;
    CU(cudaStreamWaitEvent(c->batch_aux[gi], c->batch_fork, 0), "fork wait");
    CU(launch_batch(a, g.d, g.grid, g.block, g.smem, c->batch_aux[gi]), "batch kernel");
    CU(cudaEventRecord(c->batch_join[gi], c->batch_aux[gi]), "join");
    CU(cudaStreamWaitEvent(c->stream, c->batch_join[gi], 0), "join wait");
  }
  for (size_t j = 0; j < n_jit; ++j) {
    const size_t si = B->groups.size() + j;
    CU(cudaStreamWaitEvent(c->batch_aux[si], c->batch_fork, 0), "fork wait");
    CU(launch_jit_item(B->jit[j], c->batch_aux[si]), "specialised contract");
    CU(cudaEventRecord(c->batch_join[si], c->batch_aux[si]), "join");
    CU(cudaStreamWaitEvent(c->stream, c->batch_join[si], 0), "join wait");
  }
  return PC_OK;
}

void release(pc_batch *B) {
  if (!B) return;
  destroy_graph(B);
  for (cudaStream_t st : B->aux) cudaStreamDestroy(st);
  for (cudaEvent_t ev : B->joins) cudaEventDestroy(ev);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->d_mem) cudaFree(B->d_mem);
  delete B;
}

pc_status create(size_t n, const pc_model *const *models, const pc_contract *const *contracts,
                 const uint64_t *n_paths, uint64_t seed, const pc_batch_config *config,
                 pc_batch *B, bool graph = true) {
  if (n == 0) return fail(PC_EINVAL, "empty batch");
  if (!models || !contracts || !n_paths) return fail(PC_EINVAL, "null argument");
  if (n > 0xfffffffful) return fail(PC_ELIMIT, "more than 2^32 - 1 contracts");
  if (!models[0]) return fail(PC_EINVAL, "null model");
  pc_ctx *c = models[0]->ctx;
  B->ctx = c;
  B->n = n;
  B->items.resize(n);
  B->d.resize(n);
  B->words.resize(n);
  B->tile_cost.resize(n);
  B->n_paths.assign(n_paths, n_paths + n);
  std::vector<size_t> ctl_off(n), part_off(n);
  size_t ctl_bytes = kCounterBytes, part_doubles = 0;
  for (size_t i = 0; i < n; ++i) {
    if (!models[i] || !contracts[i] || models[i]->ctx != c || contracts[i]->ctx != c)
      return fail(PC_EINVAL, "batch members must be non-null and share one context");
    if (n_paths[i] < 2) return fail(PC_EINVAL, "n_paths must be >= 2 for a standard error");
    Launch L;
    pc_status s = prepare(models[i], contracts[i], n_paths[i], 0, seed, uint32_t(i), L);
    if (s != PC_OK) return fail(s, "contract " + std::to_string(i) + ": " + pc_last_error(nullptr));
    PriceArgs &a = L.args;
    a.width = 2;
    reduction_chunks(a.n_tiles, a.chunk_tiles, a.n_chunks);
    B->d[i] = models[i]->H.d;
    B->words[i] = a.lay.words;
    B->tile_cost[i] = estimate_tile_cost(a, B->d[i]);
    B->total_tiles += a.n_tiles;
    B->total_cost += double(a.n_tiles) * B->tile_cost[i];
    ctl_off[i] = ctl_bytes;
    ctl_bytes += align256(kChunkPartOff + size_t(a.n_chunks) * 2 * sizeof(double));
    part_off[i] = part_doubles;
    part_doubles += size_t(a.n_tiles) * 2;
    B->items[i] = a;
  }
  // one allocation: items | units | counters + control blocks | partials | outputs
  const size_t items_b = align256(n * sizeof(PriceArgs));
  const size_t units_b = align256(size_t(B->total_tiles) * sizeof(BatchUnit));
  const size_t zero_b = align256(ctl_bytes);
  const size_t part_b = align256(part_doubles * sizeof(double));
  const size_t out_b = align256(n * 4 * sizeof(double));
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  CU(ctx_malloc(c, &B->d_mem, items_b + units_b + zero_b + part_b + out_b), "batch memory");
  unsigned char *base = static_cast<unsigned char *>(B->d_mem);
  B->d_items = reinterpret_cast<PriceArgs *>(base);
  B->d_units = reinterpret_cast<BatchUnit *>(base + items_b);
  B->d_zero = base + items_b + units_b;
  B->zero_bytes = zero_b;
  double *parts = reinterpret_cast<double *>(base + items_b + units_b + zero_b);
  B->d_out = reinterpret_cast<double *>(base + items_b + units_b + zero_b + part_b);
  for (size_t i = 0; i < n; ++i) {
    PriceArgs &a = B->items[i];
    a.control = B->d_zero + ctl_off[i];
    a.tile_partials = parts + part_off[i];
    a.out = B->d_out + 4 * i;
    a.out_paths = nullptr;
    a.greek_label = 0;
  }
  CU(cudaMemcpy(B->d_items, B->items.data(), n * sizeof(PriceArgs), cudaMemcpyHostToDevice), "items");
  CU(cudaMemset(B->d_out, 0, n * 4 * sizeof(double)), "outputs");
  if (graph) {
    CU(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking), "capture stream");
    CU(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming), "event");
  }
  pc_status sj = choose_jit(B, models, contracts, n_paths, seed);
  if (sj != PC_OK) return sj;
  build_groups(B);
  if (B->groups.size() > size_t(kMaxGroups)) return fail(PC_ELIMIT, "too many batch groups");
  // default: the tuner's pick on the 1024-contract synthetic portfolio
  pc_batch_config cfg{128, 128};
  if (config) cfg = *config;
  pc_status s = configure(B, cfg);
  if (s != PC_OK) return s;
  return graph ? capture(B) : PC_OK;
}

// Device milliseconds of `reps` replays (after one untimed replay).
pc_status time_replays(pc_batch *B, int reps, double &ms) {
  pc_ctx *c = B->ctx;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0), "event");
  cudaError_t e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(e, "event");
  }
  pc_status s = launch(B);
  if (s == PC_OK) {
    e = cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(B->exec, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "timed replay");
  }
  if (s == PC_OK) s = wait_stream(c);
  float t = 0.f;
  if (s == PC_OK) {
    e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) s = cuda_fail(e, "event time");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ms = double(t) / double(reps);
  return s;
}

}  // namespace

extern "C" {

pc_status pc_batch_create(size_t n, const pc_model *const *models, const pc_contract *const *contracts,
                          const uint64_t *n_paths, uint64_t seed, const pc_batch_config *config,
                          pc_batch **out) {
  if (!out) return fail(PC_EINVAL, "null output handle");
  pc_batch *B = new (std::nothrow) pc_batch;
  if (!B) return fail(PC_ENOMEM, "batch plan");
  pc_status s = create(n, models, contracts, n_paths, seed, config, B);
  if (s != PC_OK) {
    release(B);
    return s;
  }
  *out = B;
  return PC_OK;
}

pc_status pc_batch_launch(pc_batch *B) {
  if (!B || !B->exec) return fail(PC_EINVAL, "null or unconfigured batch plan");
  return launch(B);
}

pc_status pc_batch_tune(pc_batch *B, int32_t reps) {
  if (!B || !B->exec) return fail(PC_EINVAL, "null or unconfigured batch plan");
  if (reps < 1) return fail(PC_EINVAL, "reps must be >= 1");
  static const int32_t blocks[] = {128, 64};
  static const int32_t splits[] = {8, 32, 128};
  pc_batch_config best = B->cfg;
  double best_ms = -1.0;
  for (int32_t b : blocks) {
    for (int32_t u : splits) {
      const pc_batch_config cfg{b, u};
      pc_status s = configure(B, cfg);
      if (s == PC_ELIMIT) continue;  // shape does not fit this portfolio
      if (s == PC_OK) s = capture(B);
      double ms = 0.0;
      if (s == PC_OK) s = time_replays(B, reps, ms);
      if (s != PC_OK) return s;
      if (best_ms < 0.0 || ms < best_ms) {
        best_ms = ms;
        best = cfg;
      }
    }
  }
  pc_status s = configure(B, best);
  if (s == PC_OK) s = capture(B);
  if (s != PC_OK) return s;
  B->tuned = true;
  B->last_ms = best_ms;
  return PC_OK;
}

pc_status pc_batch_set_single_launch(pc_batch *B, int32_t enabled) {
  if (!B || !B->exec) return fail(PC_EINVAL, "null or unconfigured batch plan");
  if (enabled != 0 && enabled != 1) return fail(PC_EINVAL, "enabled must be 0 or 1");
  const bool was = B->single;
  B->single = enabled != 0;
  build_groups(B);
  pc_status s = configure(B, B->cfg);
  if (s == PC_OK) s = capture(B);
  if (s != PC_OK) {
    // back to the previous grouping (its configuration was valid)
    B->single = was;
    build_groups(B);
    if (configure(B, B->cfg) == PC_OK) capture(B);
    return s;
  }
  B->tuned = false;
  return PC_OK;
}

pc_status pc_batch_results(pc_batch *B, double *out_price, double *out_stderr, double *out_sums) {
  if (!B || !out_price || !out_stderr) return fail(PC_EINVAL, "null argument");
  pc_ctx *c = B->ctx;
  std::vector<double> h(B->n * 4);
  double st[5];
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  CU(cudaMemcpyAsync(h.data(), B->d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
     "result copy");
  CU(cudaMemcpyAsync(st, c->d_res, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "status copy");
  pc_status s = wait_stream(c);
  if (s != PC_OK) return s;
  int32_t status;
  std::memcpy(&status, &st[4], 4);
  s = check_status(c, status);
  if (s != PC_OK) return s;
  for (size_t i = 0; i < B->n; ++i) {
    const double N = double(B->n_paths[i]);
    if (h[4 * i + 2] != N) return fail(PC_EINVAL, "batch plan has not been launched");
  }
  for (size_t i = 0; i < B->n; ++i) {
    const double N = double(B->n_paths[i]), mean = h[4 * i] / N;
    out_price[i] = mean;
    out_stderr[i] = std::sqrt(std::max(0.0, (h[4 * i + 1] - N * mean * mean) / (N - 1.0)) / N);
    if (out_sums) {
      out_sums[3 * i] = h[4 * i];
      out_sums[3 * i + 1] = h[4 * i + 1];
      out_sums[3 * i + 2] = N;
    }
  }
  return PC_OK;
}

pc_status pc_batch_query(const pc_batch *B, pc_batch_info *info) {
  if (!B || !info) return fail(PC_EINVAL, "null argument");
  info->n_contracts = B->n;
  info->n_tiles = B->total_tiles;
  info->n_units = B->n_units;
  info->n_groups = int32_t(B->groups.size());
  info->tuned = B->tuned ? 1 : 0;
  info->config = B->cfg;
  info->paths_per_thread = B->paths_per_thread;
  info->last_ms = B->last_ms;
  info->n_specialised = B->single ? 0 : int32_t(B->jit.size());
  return PC_OK;
}

pc_status pc_batch_destroy(pc_batch *B) {
  if (!B) return fail(PC_EINVAL, "null batch plan");
  if (B->ctx) {
    cudaSetDevice(B->ctx->device);
    wait_stream(B->ctx);
  }
  release(B);
  return PC_OK;
}

pc_status pc_price_batch(size_t n, const pc_model *const *models, const pc_contract *const *contracts,
                         const uint64_t *n_paths, uint64_t seed, double *out_price,
                         double *out_stderr) {
  if (n == 0) return PC_OK;
  if (!out_price || !out_stderr) return fail(PC_EINVAL, "null argument");
  // a plan without a graph: its groups launched once, straight away
  pc_batch *B = new (std::nothrow) pc_batch;
  if (!B) return fail(PC_ENOMEM, "batch plan");
  pc_status s = create(n, models, contracts, n_paths, seed, nullptr, B, false);
  if (s == PC_OK) s = launch_direct(B);
  if (s == PC_OK) s = pc_batch_results(B, out_price, out_stderr, nullptr);
  pc_batch_destroy(B);
  return s;
}

}  // extern "C"
