// pc_capi.cpp -- the extern "C" entry points declared in include/pc.h.
//
// Host orchestration only: argument checks, load-time compilation of payoff
// programs, model setup, device uploads, kernel launches on the context's
// stream and bounded waits.  Every step of the per-path computation runs in
// the kernels of pc_kernels.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include "pc_handles.h"
#include "pc_internal.h"

using namespace pc;

namespace {
thread_local std::string tl_err;
std::atomic<uint64_t> g_model_ids{1};
}  // namespace

namespace pc {

pc_status fail(pc_status s, const std::string &m) {
  tl_err = m;
  return s;
}

pc_status cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

// Wait for the stream with a wall-clock limit.
pc_status wait_stream(pc_ctx *c) {
  const auto t_start = std::chrono::steady_clock::now();
  int spins = 0;
  for (;;) {
    cudaError_t e = cudaStreamQuery(c->stream);
    if (e == cudaSuccess) return PC_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "stream");
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (el > c->timeout_s) return fail(PC_ETIMEOUT, "device did not finish within the context's limit");
    if (++spins > 2000) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

cudaError_t ctx_malloc(pc_ctx *c, void **p, size_t bytes) {
  if (c->fail_allocs > 0) {
    --c->fail_allocs;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t ctx_alloc(pc_ctx *c, void **p, size_t bytes, bool &pooled) {
  pooled = c->pool != nullptr;
  if (c->fail_allocs > 0) {
    --c->fail_allocs;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  if (pooled) return cudaMallocFromPoolAsync(p, bytes, c->pool, c->stream);
  return cudaMalloc(p, bytes);
}

void ctx_free(pc_ctx *c, void *p, bool pooled) {
  if (!p) return;
  if (pooled) {
    cudaFreeAsync(p, c->stream);
  } else {
    cudaStreamSynchronize(c->stream);
    cudaFree(p);
  }
}

cudaError_t jit_occupancy(pc_ctx *c, const void *kern, int block, size_t smem, int &blocks) {
  std::lock_guard<std::mutex> g(c->jit_mu);
  const auto key = std::make_pair(kern, smem * 1024 + size_t(block));
  auto it = c->jit_occ.find(key);
  if (it != c->jit_occ.end()) {
    blocks = it->second;
    return cudaSuccess;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, block, smem);
  if (e == cudaSuccess) c->jit_occ.emplace(key, blocks);
  return e;
}

template <typename T>
pc_status upload(const std::vector<T> &v, char *base, size_t &off, const T *&dst, cudaStream_t s) {
  off = (off + 255) & ~size_t(255);
  dst = reinterpret_cast<const T *>(base + off);
  if (!v.empty())
    CU(cudaMemcpyAsync(base + off, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s), "upload");
  off += v.size() * sizeof(T);
  return PC_OK;
}

template <typename T>
size_t padded(const std::vector<T> &v) { return ((v.size() * sizeof(T)) + 255) & ~size_t(255); }

Layout make_layout(const Program &p, const ModelHost &H, int32_t win) {
  Layout L{};
  L.stack = p.frame_slots;
  L.off_bstack = L.stack;
  L.off_cache = L.off_bstack + H.bstack * H.d;  // caches are in registers: no words
  L.off_win = L.off_cache;
  L.win = win;
  // slot of ordinal o is o & (win - 1); when the whole grid fits (n < win)
  // that is o itself, so only slots 0..n are ever touched
  L.words = L.off_win + std::min(win, H.n + 1) * H.d;
  return L;
}

pc_status ensure_partials(pc_ctx *c, size_t doubles) {
  if (doubles <= c->partial_cap) return PC_OK;
  CU(cudaStreamSynchronize(c->stream), "sync");
  if (c->d_partials) cudaFree(c->d_partials);
  c->d_partials = nullptr;
  c->partial_cap = 0;
  size_t cap = std::max<size_t>(doubles, 1 << 16);
  CU(ctx_malloc(c, reinterpret_cast<void **>(&c->d_partials), cap * sizeof(double)), "partials");
  c->partial_cap = cap;
  return PC_OK;
}

// Constant-pool floats of a program, rounded up to whole 16-byte words.
size_t pool_padded(const Program &p) { return (p.pool.size() + 3) & ~size_t(3); }

// Highest underlying label a program reads (-1 if none).
int32_t max_label(const Program &p) {
  int32_t top = -1;
  for (const XInsn &I : p.code) {
    const uint32_t op = I.opa & 0xffu;
    if (op == X_MODEL || op == X_MODEL_MULK || op == X_MODEL_DIVK) {
      top = std::max(top, int32_t(I.opa >> 8));
    } else if (op == X_LRED || op == X_LANY) {
      const uint32_t n = ((I.opa >> 8 >> 8) & 3u) + 1;
      for (uint32_t i = 0; i < n; ++i) top = std::max(top, int32_t((I.opa >> 8 >> (10 + 2 * i)) & 3u));
    }
  }
  return top;
}

pc_status window_for(const pc_model *m, const pc_contract *k, int32_t &win) {
  auto *kc = const_cast<pc_contract *>(k);
  std::lock_guard<std::mutex> g(kc->mu);
  auto key = std::make_pair(m->id, uint64_t(0));
  auto it = kc->win_cache.find(key);
  if (it != kc->win_cache.end()) { win = it->second; return PC_OK; }
  // labels must exist in the model
  const int32_t top = max_label(k->prog);
  if (top >= m->H.d)
    return fail(PC_ERANGE, "program observes label " + std::to_string(top) + " but the model has " +
                               std::to_string(m->H.d) + " underlyings");
  std::string err;
  pc_status s = analyse_program(k->prog, m->H.t_now, m->H.n, m->H.n_hist, win, err);
  if (s != PC_OK) return fail(s, err);
  kc->win_cache[key] = win;
  return PC_OK;
}

// Block size (128, 64 or 32 threads) that keeps the most warps resident per
// SM given the program's shared-memory footprint; 0 if none fits.  Without
// `memoise` the occupancy queries store nothing (no host allocation).
int pick_block(const Program &p, int words, int max_smem, int d, size_t &smem, bool memoise = true) {
  int best = 0, best_warps = 0;
  size_t best_smem = 0;
  for (int b = kBlock; b >= 32; b /= 2) {
    const size_t sm = price_smem_bytes(p.code.size(), pool_padded(p), words, b);
    if (sm + kStaticSmemReserve > size_t(max_smem)) continue;
    const int warps = price_blocks_per_sm(d, b, sm, false, memoise) * (b / 32);
    if (warps > best_warps) {
      best = b;
      best_warps = warps;
      best_smem = sm;
    }
  }
  smem = best ? best_smem : price_smem_bytes(p.code.size(), pool_padded(p), words, 32);
  return best;
}

pc_status prepare(const pc_model *m, const pc_contract *k, uint64_t n_paths, uint64_t offset,
                  uint64_t seed, uint32_t stream, Launch &L, bool allow_hbm) {
  if (!m || !k) return fail(PC_EINVAL, "null model or contract");
  if (m->ctx != k->ctx) return fail(PC_EINVAL, "model and contract belong to different contexts");
  if (n_paths == 0) return fail(PC_EINVAL, "n_paths must be >= 1");
  if (n_paths > (uint64_t(1) << 40)) return fail(PC_ELIMIT, "n_paths exceeds 2^40");
  int32_t win = 1;
  pc_status s = window_for(m, k, win);
  if (s != PC_OK) return s;
  pc_ctx *c = m->ctx;
  const int mode = allow_hbm ? c->window_mode : PC_WINDOW_SHARED;
  Layout lay = make_layout(k->prog, m->H, win);
  int bpsm = 0;
  bool hbm = mode == PC_WINDOW_HBM;
  if (!hbm) {
    L.block = win <= PC_MAX_WINDOW ? pick_block(k->prog, lay.words, c->max_smem, m->H.d, L.smem) : 0;
    bpsm = L.block ? price_blocks_per_sm(m->H.d, L.block, L.smem, false) : 0;
    const int warps = bpsm * L.block / 32;
    if (mode == PC_WINDOW_AUTO && (!L.block || warps < 8)) hbm = true;
  }
  if (hbm) {
    // shared region without the window; the window is a column of the
    // context's HBM window buffer per thread of the launch
    lay.off_win = lay.off_cache;
    lay.words = lay.off_win;
    L.block = kBlock;
    L.smem = price_smem_bytes(k->prog.code.size(), pool_padded(k->prog), lay.words, L.block);
    if (L.smem + kStaticSmemReserve > size_t(c->max_smem)) {
      L.block = 32;
      L.smem = price_smem_bytes(k->prog.code.size(), pool_padded(k->prog), lay.words, L.block);
    }
    bpsm = price_blocks_per_sm(m->H.d, L.block, L.smem, true);
    L.hbm_window = true;
  } else if (!L.block) {
    if (win > PC_MAX_WINDOW)
      return fail(PC_ERANGE, "program looks back " + std::to_string(win / 2) + "+ dates; this entry point "
                             "keeps at most " + std::to_string(PC_MAX_WINDOW) + " in shared memory");
    return fail(PC_ELIMIT, "program + per-path state need " + std::to_string(L.smem) +
                               " bytes of shared memory for a 32-thread block; the device offers " +
                               std::to_string(c->max_smem));
  }
  const uint64_t n_tiles = (n_paths + kTilePaths - 1) / kTilePaths;
  PriceArgs &a = L.args;
  a.prog = k->d_code;
  a.n_insn = int32_t(k->prog.code.size());
  a.n_pool = int32_t(pool_padded(k->prog));
  a.m = m->dev;
  a.lay = lay;
  a.n_paths = n_paths;
  a.path_offset = offset;
  a.key0 = uint32_t(seed);
  a.key1 = uint32_t(seed >> 32);
  philox_round_keys(seed, a.rk);
  a.stream = stream;
  a.n_tiles = n_tiles;
  a.status = reinterpret_cast<int32_t *>(c->d_res + 4);
  if (bpsm < 1) return fail(PC_ELIMIT, "kernel cannot be resident with this shared-memory footprint");
  const uint64_t warps_per_block = uint64_t(L.block) / 32;
  const uint64_t need = (n_tiles + warps_per_block - 1) / warps_per_block;
  L.grid = int(std::min<uint64_t>(uint64_t(c->sm_count) * bpsm, need));
  return PC_OK;
}

// Point the launch's window at the context's HBM window buffer (grown to
// grid * block threads x win * d slots).
pc_status bind_hbm_window(pc_ctx *c, Launch &L, int d) {
  const size_t threads = size_t(L.grid) * size_t(L.block);
  const size_t slots = threads * size_t(L.args.lay.win) * size_t(d);
  if (slots > c->gwin_cap) {
    CU(cudaStreamSynchronize(c->stream), "sync");
    if (c->d_gwin) cudaFree(c->d_gwin);
    c->d_gwin = nullptr;
    c->gwin_cap = 0;
    CU(ctx_malloc(c, reinterpret_cast<void **>(&c->d_gwin), slots * sizeof(float2)), "HBM window");
    c->gwin_cap = slots;
  }
  L.args.lay.gwin = c->d_gwin;
  L.args.lay.gstride = int64_t(threads);
  return PC_OK;
}

// Sensitivity launch for underlying `label`: the pricing launch set-up with
// three physical slots per program value and an extra window of X = L W.
pc_status run_greeks(const pc_model *m, const pc_contract *k, uint64_t n_paths, uint64_t offset,
                     uint64_t seed, int label, double *d_out, float *d_paths) {
  Launch L;
  pc_status s = prepare(m, k, n_paths, offset, seed, 0, L);
  if (s != PC_OK) return s;
  pc_ctx *c = m->ctx;
  Layout lay = L.args.lay;
  const int d = m->H.d;
  lay.stack = 3 * k->prog.frame_slots;
  lay.off_bstack = lay.stack;
  lay.off_cache = lay.off_bstack + m->H.bstack * d;
  lay.off_win = lay.off_cache;
  lay.off_xwin = lay.off_win + lay.win * d;
  lay.words = lay.off_xwin + lay.win * d;
  int block = 0, best_warps = 0;
  size_t smem = 0;
  for (int b = kBlock; b >= 32; b /= 2) {
    const size_t sm = price_smem_bytes(k->prog.code.size(), pool_padded(k->prog), lay.words, b);
    if (sm + kStaticSmemReserve > size_t(c->max_smem)) continue;
    const int warps = greeks_blocks_per_sm(d, b, sm) * (b / 32);
    if (warps > best_warps) { block = b; best_warps = warps; smem = sm; }
  }
  if (!block) return fail(PC_ELIMIT, "program + per-path state with sensitivities exceed shared memory");
  s = ensure_partials(c, size_t(L.args.n_tiles) * 6);
  if (s != PC_OK) return s;
  PriceArgs a = L.args;
  a.lay = lay;
  a.width = 6;
  reduction_chunks(a.n_tiles, a.chunk_tiles, a.n_chunks);
  a.tile_partials = c->d_partials;
  a.control = c->d_control;
  a.out = d_out;
  a.out_paths = d_paths;
  a.greek_label = label;
  const uint64_t need = (a.n_tiles + block / 32 - 1) / (block / 32);
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  if (c->jit && jit_eligible(k)) {
    // the contract's run-time specialised tangent kernel (same arguments,
    // shared-memory layout and block)
    cudaKernel_t jk = nullptr;
    s = jit_kernel(k, d, kJitGreeks + (d_paths != nullptr ? 1 : 0), block, jk);
    if (s != PC_OK) return s;
    const void *kern = reinterpret_cast<const void *>(jk);
    int nb = 0;
    CU(jit_occupancy(c, kern, block, smem, nb), "jit occupancy");
    if (nb < 1) return fail(PC_ELIMIT, "specialised sensitivity kernel cannot be resident");
    const int jgrid = int(std::min<uint64_t>(uint64_t(c->sm_count) * nb, need));
    void *args[] = {&a};
    CU(cudaLaunchKernel(kern, dim3(jgrid), dim3(block), args, smem, c->stream), "specialised sensitivity kernel");
    return PC_OK;
  }
  const int grid = int(std::min<uint64_t>(uint64_t(c->sm_count) * best_warps / (block / 32), need));
  CU(launch_greeks(a, grid, block, smem, c->stream), "sensitivity kernel");
  return PC_OK;
}

// Kind bits of the launch's specialised pricing kernel beyond the variant:
// the window of dates in HBM, or a window of one date (a program that reads
// no date behind the frontier), which the kernel keeps in registers, then
// with the context's choice of two path pairs a lane.
int jit_window_kind(const pc_ctx *c, const Launch &L) {
  if (L.hbm_window) return kJitHbm;
  if (L.args.lay.win != 1) return 0;
  // automatic: two pairs where a path walks many dates (the daily barrier's
  // 365: 6.84 -> 6.49 ms at 2^22 paths); a few dates gain nothing (5 dates:
  // 0.069 ms either way), the tile loop and the reduction dominate there
  const bool two = c->jit_pairs == 2 || (c->jit_pairs == 0 && L.args.m.n >= kJitPairsMinDates);
  return kJitWinRegs | (two ? kJitPairs2 : 0);
}

// The specialised evaluator keeps its operand stack in registers, and with
// kJitWinRegs the window too: drop those words from the per-thread shared
// region of the launch.  Returns the launch's dynamic shared memory.
// With two path pairs a lane the bridge stack holds both pairs' values per
// level (twice the words), and the block is re-chosen for the most resident
// warps that shared memory allows.
size_t jit_layout(const pc_ctx *c, const pc_contract *k, Launch &L, int bits) {
  Layout &lay = L.args.lay;
  const int shift = lay.off_bstack;
  lay.stack = 0;
  lay.off_bstack -= shift;
  lay.off_cache -= shift;
  lay.off_win -= shift;
  lay.words -= shift;
  if (bits & kJitWinRegs) lay.words = lay.off_win;
  if (bits & kJitPairs2) {
    lay.words = lay.off_bstack + 2 * (lay.off_cache - lay.off_bstack);
    int best = 0, best_warps = 0;
    for (int b = kBlock; b >= 32; b /= 2) {
      const size_t sm = price_smem_bytes(k->prog.code.size(), pool_padded(k->prog), lay.words, b);
      if (sm + kStaticSmemReserve > size_t(c->max_smem)) continue;
      const size_t per = sm + kJitStaticSmem + size_t(c->smem_reserve);
      const int blocks = c->sm_smem > 0 ? std::min<int>(32, int(size_t(c->sm_smem) / per)) : 1;
      if (blocks * (b / 32) > best_warps) {
        best_warps = blocks * (b / 32);
        best = b;
      }
    }
    if (best) L.block = best;
  }
  return price_smem_bytes(k->prog.code.size(), pool_padded(k->prog), lay.words, L.block);
}

// Resident blocks per SM (of kBlock threads, the block the kernel's bound
// is written for) the specialised pricing kernel's register bound is set
// for: the default, or fewer when the launch's shared memory allows no more
// warps (the kernel may then use the registers those blocks leave).  The
// kernel's own static shared memory is a few words (kJitStaticSmem bounds it).
int jit_min_blocks(const pc_ctx *c, size_t smem, int block) {
  if (c->sm_smem <= 0) return kJitMinBlocks;
  const size_t per = smem + kJitStaticSmem + size_t(c->smem_reserve);
  const int warps = int(size_t(c->sm_smem) / per) * (block / 32);
  return std::max(1, std::min(kJitMinBlocks, warps / (kBlock / 32)));
}

pc_status run_price(const pc_model *m, const pc_contract *k, uint64_t n_paths, uint64_t offset,
                    uint64_t seed, uint32_t stream, double *d_out, float *d_payoffs) {
  Launch L;
  pc_status s = prepare(m, k, n_paths, offset, seed, stream, L, true);
  if (s != PC_OK) return s;
  pc_ctx *c = m->ctx;
  s = ensure_partials(c, size_t(L.args.n_tiles) * 2);
  if (s != PC_OK) return s;
  L.args.width = 2;
  reduction_chunks(L.args.n_tiles, L.args.chunk_tiles, L.args.n_chunks);
  L.args.tile_partials = c->d_partials;
  L.args.control = c->d_control;
  L.args.out = d_out;
  L.args.out_paths = d_payoffs;
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  if (c->jit && jit_eligible(k)) {
    // the contract's run-time specialised kernel (same arguments and shape)
    cudaKernel_t jk = nullptr;
    const int wk = jit_window_kind(c, L);
    const size_t smem = jit_layout(c, k, L, wk);
    s = jit_kernel(k, m->H.d, (d_payoffs != nullptr ? kJitPriceWrite : kJitPrice) | wk, L.block, jk,
                   jit_min_blocks(c, smem, L.block));
    if (s != PC_OK) return s;
    const void *kern = reinterpret_cast<const void *>(jk);
    int nb = 0;
    CU(jit_occupancy(c, kern, L.block, smem, nb), "jit occupancy");
    if (nb < 1) return fail(PC_ELIMIT, "specialised kernel cannot be resident");
    const uint64_t wpb = uint64_t(L.block) / 32;
    // a warp takes a tile, or a pair of tiles with two path pairs a lane
    const uint64_t units = (wk & kJitPairs2) ? (L.args.n_tiles + 1) / 2 : L.args.n_tiles;
    const int grid = int(std::min<uint64_t>(uint64_t(c->sm_count) * nb, (units + wpb - 1) / wpb));
    if (L.hbm_window) {
      // the HBM window holds a column per thread of this launch's grid
      L.grid = grid;
      s = bind_hbm_window(c, L, m->H.d);
      if (s != PC_OK) return s;
    }
    void *args[] = {&L.args};
    CU(cudaLaunchKernel(kern, dim3(grid), dim3(L.block), args, smem, c->stream), "specialised price kernel");
    return PC_OK;
  }
  if (L.hbm_window) {
    s = bind_hbm_window(c, L, m->H.d);
    if (s != PC_OK) return s;
  }
  CU(launch_price(L.args, L.grid, L.block, L.smem, c->stream), "price kernel");
  return PC_OK;
}

pc_status check_status(pc_ctx *c, int32_t status) {
  if (status == 0) return PC_OK;
  int32_t zero = 0;
  cudaMemcpyAsync(reinterpret_cast<int32_t *>(c->d_res + 4), &zero, 4, cudaMemcpyHostToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  return fail(PC_EDEVICE, "kernel raised its status word (" + std::to_string(status) + ")");
}

}  // namespace pc

extern "C" {

pc_status pc_price_noalloc(const pc_model *m, const pc_contract *k, uint64_t n_paths,
                           uint64_t path_offset, uint64_t seed, uint32_t stream, double *d_out) {
  if (!m || !k || !d_out) return fail(PC_EINVAL, "null model, contract or d_out");
  if (m->ctx != k->ctx) return fail(PC_EINVAL, "model and contract belong to different contexts");
  if (n_paths == 0) return fail(PC_EINVAL, "n_paths must be >= 1");
  if (n_paths > PC_NOALLOC_MAX_PATHS)
    return fail(PC_ELIMIT, "pc_price_noalloc prices at most PC_NOALLOC_MAX_PATHS (2^24) paths per call");
  const ModelHost &H = m->H;
  if (max_label(k->prog) >= H.d)
    return fail(PC_ERANGE, "program observes a label the model does not have");
  pc_ctx *c = m->ctx;
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  // the window: from the contract's cache when an allocating call resolved
  // it for this model already (a lookup, no insertion), else by the same
  // analysis without storing it
  int32_t win = 0;
  {
    auto *kc = const_cast<pc_contract *>(k);
    std::lock_guard<std::mutex> g(kc->mu);
    const auto it = kc->win_cache.find(std::make_pair(m->id, uint64_t(0)));
    if (it != kc->win_cache.end()) {
      win = it->second;
    } else {
      const char *why = "";
      auto on_fail = [&](pc_status st, int64_t, int64_t) {
        why = st == PC_ELIMIT ? "program too long to analyse (loop trip counts)"
                              : "a model or payoff time is outside the model's grid";
      };
      TimeWalk<decltype(on_fail)> walk{k->prog.code.data(), H.t_now, H.n, H.n_hist, on_fail};
      walk.run(0, k->prog.code.size(), 0);
      if (walk.st != PC_OK) return fail(walk.st, why);
      win = walk.window();
    }
  }
  if (win > PC_MAX_WINDOW)
    return fail(PC_ERANGE, "program looks back further than PC_MAX_WINDOW dates; pc_price_noalloc keeps "
                           "the window of dates in shared memory only");
  const Layout lay = make_layout(k->prog, H, win);
  size_t smem = 0;
  const int block = pick_block(k->prog, lay.words, c->max_smem, H.d, smem, false);
  if (!block) return fail(PC_ELIMIT, "program + per-path state exceed the device's shared memory per block");
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  CU(noalloc_scratch(&scratch, &scratch_bytes), "scratch lookup");
  const uint64_t n_tiles = (n_paths + kTilePaths - 1) / kTilePaths;
  if (kNoAllocCounterBytes + n_tiles * 2 * sizeof(double) > scratch_bytes)
    return fail(PC_ELIMIT, "request exceeds the fixed scratch array");
  const int bpsm = price_blocks_per_sm(H.d, block, smem, false, false);
  if (bpsm < 1) return fail(PC_ELIMIT, "kernel cannot be resident with this shared-memory footprint");
  PriceArgs a{};
  a.prog = k->d_code;
  a.n_insn = int32_t(k->prog.code.size());
  a.n_pool = int32_t(pool_padded(k->prog));
  a.m = m->dev;
  a.lay = lay;
  a.n_paths = n_paths;
  a.path_offset = path_offset;
  a.key0 = uint32_t(seed);
  a.key1 = uint32_t(seed >> 32);
  philox_round_keys(seed, a.rk);
  a.stream = stream;
  a.n_tiles = n_tiles;
  a.width = 2;
  reduction_chunks(n_tiles, a.chunk_tiles, a.n_chunks);
  a.control = static_cast<unsigned char *>(scratch);
  a.tile_partials = reinterpret_cast<double *>(static_cast<char *>(scratch) + kNoAllocCounterBytes);
  a.out = d_out;
  a.out_paths = nullptr;
  a.status = reinterpret_cast<int32_t *>(c->d_res + 4);
  const uint64_t need = (n_tiles + block / 32 - 1) / (block / 32);
  const int grid = int(std::min<uint64_t>(uint64_t(c->sm_count) * bpsm, need));
  CU(cudaMemsetAsync(a.control, 0, kNoAllocCounterBytes, c->stream), "counter reset");
  CU(launch_price(a, grid, block, smem, c->stream), "price kernel");
  return PC_OK;
}


pc_status pc_set_timeout(pc_ctx *c, double seconds) {
  if (!c) return fail(PC_EINVAL, "null context");
  if (!(seconds > 0.0) || !std::isfinite(seconds)) return fail(PC_EINVAL, "the limit must be a positive number of seconds");
  c->timeout_s = seconds;
  return PC_OK;
}

pc_status pc_debug_fail_allocations(pc_ctx *c, int32_t count) {
  if (!c) return fail(PC_EINVAL, "null context");
  if (count < 0) return fail(PC_EINVAL, "count must be >= 0");
  c->fail_allocs = count;
  return PC_OK;
}

pc_status pc_debug_set_status(pc_ctx *c, int32_t value) {
  if (!c) return fail(PC_EINVAL, "null context");
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  CU(cudaMemcpyAsync(reinterpret_cast<int32_t *>(c->d_res + 4), &value, 4, cudaMemcpyHostToDevice, c->stream),
     "status write");
  return wait_stream(c);
}

const char *pc_last_error(const pc_ctx *) { return tl_err.c_str(); }

pc_status pc_create(pc_ctx **out, int device, void *cuda_stream) {
  if (!out) return fail(PC_EINVAL, "out is null");
  int n = 0;
  CU(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(PC_EINVAL, "no such CUDA device");
  cudaDeviceProp prop{};
  CU(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3)
    return fail(PC_ECUDA, std::string("kernels are built for sm_103a; device is ") + prop.name +
                              " (sm_" + std::to_string(prop.major) + std::to_string(prop.minor) + ")");
  CU(cudaSetDevice(device), "cudaSetDevice");
  pc_ctx *c = new (std::nothrow) pc_ctx();
  if (!c) return fail(PC_ENOMEM, "context");
  c->device = device;
  c->sm_count = prop.multiProcessorCount;
  c->max_smem = max_dynamic_smem();
  CU(cudaDeviceGetAttribute(&c->sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device), "device attribute");
  CU(cudaDeviceGetAttribute(&c->smem_reserve, cudaDevAttrReservedSharedMemoryPerBlock, device), "device attribute");
  if (const char *t = std::getenv("PC_TIMEOUT_S")) c->timeout_s = std::max(1.0, std::atof(t));
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    c->own_stream = true;
  }
  if (e == cudaSuccess) {
    // a memory pool of the context's own, keeping freed memory (contracts
    // are loaded and dropped often): stream-ordered, no device-wide sync
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
      uint64_t keep = ~uint64_t(0);
      cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      c->pool = nullptr;
      cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&c->h_res), 16 * sizeof(double), 0);
  if (e == cudaSuccess) {
    c->stage_words = 16384;
    e = cudaHostAlloc(reinterpret_cast<void **>(&c->h_stage), 2 * c->stage_words * 4, 0);
  }
  for (int h = 0; h < 2 && e == cudaSuccess; ++h) e = cudaEventCreateWithFlags(&c->stage_ev[h], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_res, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_res, 0, 8 * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_gout, PC_MAX_UNDERLYINGS * 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_control, kControlBytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_control, 0, kControlBytes, c->stream);
  if (e == cudaSuccess) {
    // pc_price_noalloc's fixed scratch array: looking its address up here
    // loads the kernels' module on this device, which reserves the array,
    // when the context is created rather than inside a pc_price_noalloc call
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    e = noalloc_scratch(&scratch, &scratch_bytes);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    if (c->d_control) cudaFree(c->d_control);
    if (c->d_gout) cudaFree(c->d_gout);
    if (c->d_res) cudaFree(c->d_res);
    for (cudaEvent_t ev : c->stage_ev)
      if (ev) cudaEventDestroy(ev);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->h_res) cudaFreeHost(c->h_res);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return cuda_fail(e, "context setup");
  }
  *out = c;
  return PC_OK;
}

pc_status pc_destroy(pc_ctx *c) {
  if (!c) return fail(PC_EINVAL, "null context");
  if (c->live_objects) return fail(PC_EINVAL, "destroy the context's models and contracts first");
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->d_partials) cudaFree(c->d_partials);
  if (c->d_control) cudaFree(c->d_control);
  if (c->d_gwin) cudaFree(c->d_gwin);
  if (c->d_tape) cudaFree(c->d_tape);
  jit_release(c);
  if (c->d_gout) cudaFree(c->d_gout);
  if (c->d_res) cudaFree(c->d_res);
  for (cudaEvent_t ev : c->stage_ev)
    if (ev) cudaEventDestroy(ev);
  for (cudaStream_t st : c->batch_aux) cudaStreamDestroy(st);
  for (cudaEvent_t ev : c->batch_join) cudaEventDestroy(ev);
  if (c->batch_fork) cudaEventDestroy(c->batch_fork);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->h_res) cudaFreeHost(c->h_res);
  if (c->pool) cudaMemPoolDestroy(c->pool);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return PC_OK;
}

pc_status pc_model_create(pc_ctx *c, const pc_model_desc *desc, pc_model **out) {
  if (!c || !desc || !out) return fail(PC_EINVAL, "null argument");
  try {
    pc_model *m = new pc_model();
    std::string err;
    pc_status s = build_model(*desc, m->H, err);
    if (s != PC_OK) {
      delete m;
      return fail(s, err);
    }
    const ModelHost &H = m->H;
    size_t bytes = padded(H.date_ops) + padded(H.ops) + padded(H.A) + padded(H.B) +
                   padded(H.disc) + padded(H.sval) + padded(H.tau) + padded(H.Lf) +
                   padded(H.sig) + 256;
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    cudaError_t e = ctx_malloc(c, &m->d_mem, bytes);
    if (e != cudaSuccess) {
      delete m;
      return cuda_fail(e, "model tables");
    }
    char *base = static_cast<char *>(m->d_mem);
    size_t off = 0;
    ModelDev &D = m->dev;
    pc_status u = PC_OK;
    if (u == PC_OK) u = upload(H.date_ops, base, off, D.date_ops, c->stream);
    if (u == PC_OK) u = upload(H.ops, base, off, D.ops, c->stream);
    if (u == PC_OK) u = upload(H.A, base, off, D.A, c->stream);
    if (u == PC_OK) u = upload(H.B, base, off, D.B, c->stream);
    if (u == PC_OK) u = upload(H.disc, base, off, D.disc, c->stream);
    if (u == PC_OK) u = upload(H.sval, base, off, D.sval, c->stream);
    if (u == PC_OK) u = upload(H.tau, base, off, D.tau, c->stream);
    if (u == PC_OK) u = upload(H.Lf, base, off, D.L, c->stream);
    if (u == PC_OK) u = upload(H.sig, base, off, D.sig, c->stream);
    if (u == PC_OK) {
      cudaError_t e2 = cudaStreamSynchronize(c->stream);
      if (e2 != cudaSuccess) u = cuda_fail(e2, "model upload");
    }
    if (u != PC_OK) {
      cudaFree(m->d_mem);
      delete m;
      return u;
    }
    for (size_t i = 0; i < H.B.size() && i < 16; ++i) D.Bv[i] = H.B[i];
    for (int i = 0; i < H.d; ++i) D.S0v[i] = H.sval[size_t(H.n_hist) * H.d + i];
    D.d = H.d;
    D.n = H.n;
    D.n_hist = H.n_hist;
    D.t_now = H.t_now;
    D.n_levels = H.n_levels;
    D.bstack = H.bstack;
    m->ctx = c;
    m->id = g_model_ids.fetch_add(1);
    ++c->live_objects;
    *out = m;
    return PC_OK;
  } catch (const std::bad_alloc &) {
    return fail(PC_ENOMEM, "host allocation");
  } catch (...) {
    return fail(PC_EINVAL, "unexpected error in pc_model_create");
  }
}

pc_status pc_model_query(const pc_model *m, pc_model_info *info) {
  if (!m || !info) return fail(PC_EINVAL, "null argument");
  const ModelHost &H = m->H;
  info->d = H.d;
  info->n_dates = H.n;
  info->n_hist = H.n_hist;
  info->t_now = H.t_now;
  info->bridge_levels = H.n_levels;
  info->bridge_stack = H.bstack;
  // the n d normals of a path in counter order: four per Philox block
  const int32_t blocks = int32_t((int64_t(H.ops.size()) * H.d + 3) / 4);
  info->philox_blocks = blocks;
  info->box_muller_pairs = 2 * blocks;
  return PC_OK;
}

pc_status pc_model_destroy(pc_model *m) {
  if (!m) return fail(PC_EINVAL, "null model");
  cudaSetDevice(m->ctx->device);
  cudaStreamSynchronize(m->ctx->stream);
  cudaFree(m->d_mem);
  --m->ctx->live_objects;
  delete m;
  return PC_OK;
}

pc_status pc_verify_payoff(const uint32_t *bytecode, size_t n_words, const double *consts,
                           size_t n_consts, const int32_t *template_params, size_t n_params,
                           pc_program_info *info) {
  try {
    Program p;
    std::string err;
    pc_status s = compile_program(bytecode, n_words, consts, n_consts, template_params, n_params,
                                  0, 1, false, p, err);
    if (s != PC_OK) return fail(s, err);
    if (info) *info = p.info;
    return PC_OK;
  } catch (const std::bad_alloc &) {
    return fail(PC_ENOMEM, "host allocation");
  } catch (...) {
    return fail(PC_EINVAL, "unexpected error in pc_verify_payoff");
  }
}

pc_status pc_load_payoffs(pc_ctx *c, size_t n, const uint32_t *words, const size_t *word_off,
                          const double *consts, const size_t *const_off, const int32_t *params,
                          const size_t *param_off, int32_t p1, int32_t p2, pc_contract **out) {
  if (!c || !out || !word_off || !const_off || !param_off || (n && !words)) return fail(PC_EINVAL, "null argument");
  for (size_t i = 0; i < n; ++i)
    if (word_off[i + 1] < word_off[i] || const_off[i + 1] < const_off[i] || param_off[i + 1] < param_off[i])
      return fail(PC_EINVAL, "offsets must be non-decreasing");
  if ((const_off[n] > const_off[0] && !consts) || (param_off[n] > param_off[0] && !params))
    return fail(PC_EINVAL, "null literals or parameters");
  std::vector<pc_contract *> done;
  done.reserve(n);
  for (size_t i = 0; i < n; ++i) {
    pc_contract *k = nullptr;
    const pc_status s = pc_load_payoff(c, words + word_off[i], word_off[i + 1] - word_off[i],
                                       consts ? consts + const_off[i] : nullptr, const_off[i + 1] - const_off[i],
                                       params ? params + param_off[i] : nullptr, param_off[i + 1] - param_off[i],
                                       p1, p2, &k);
    if (s != PC_OK) {
      const std::string msg = "program " + std::to_string(i) + ": " + pc_last_error(nullptr);
      for (pc_contract *d : done) pc_contract_destroy(d);
      return fail(s, msg);
    }
    done.push_back(k);
  }
  for (size_t i = 0; i < n; ++i) out[i] = done[i];
  return PC_OK;
}

pc_status pc_load_payoff(pc_ctx *c, const uint32_t *bytecode, size_t n_words, const double *consts,
                         size_t n_consts, const int32_t *template_params, size_t n_params,
                         int32_t p1, int32_t p2, pc_contract **out) {
  if (!c || !out) return fail(PC_EINVAL, "null argument");
  try {
    pc_contract *k = new pc_contract();
    // the compiler's inputs as words: the cache key
    std::vector<uint32_t> key;
    key.reserve(n_words + 2 * n_consts + n_params + 5);
    key.push_back(uint32_t(n_words));
    key.push_back(uint32_t(n_consts));
    key.push_back(uint32_t(n_params));
    key.push_back(uint32_t(p1));
    key.push_back(uint32_t(p2));
    if (bytecode) key.insert(key.end(), bytecode, bytecode + n_words);
    for (size_t i = 0; consts && i < n_consts; ++i) {
      uint64_t b;
      std::memcpy(&b, consts + i, 8);
      key.push_back(uint32_t(b));
      key.push_back(uint32_t(b >> 32));
    }
    for (size_t i = 0; template_params && i < n_params; ++i) key.push_back(uint32_t(template_params[i]));
    uint64_t h = 1469598103934665603ull;  // FNV-1a
    for (uint32_t w : key)
      for (int b = 0; b < 4; ++b) h = (h ^ ((w >> (8 * b)) & 0xffu)) * 1099511628211ull;
    bool hit = false;
    {
      std::lock_guard<std::mutex> g(c->load_mu);
      auto range = c->program_cache.equal_range(h);
      for (auto it = range.first; it != range.second; ++it)
        if (it->second.first == key) {
          k->prog = it->second.second;
          hit = true;
          break;
        }
    }
    if (!hit) {
      std::string err;
      pc_status s = compile_program(bytecode, n_words, consts, n_consts, template_params, n_params,
                                    p1, p2, true, k->prog, err);
      if (s != PC_OK) {
        delete k;
        return fail(s, err);
      }
      std::lock_guard<std::mutex> g(c->load_mu);
      if (c->program_cache.size() >= 4096) c->program_cache.clear();
      c->program_cache.emplace(h, std::make_pair(std::move(key), k->prog));
    }
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    // program then constant pool (padded to whole 16-byte words), one buffer
    const size_t code_words = k->prog.code.size() * 4;
    k->image.assign(code_words + pool_padded(k->prog), 0u);
    std::memcpy(k->image.data(), k->prog.code.data(), code_words * 4);
    std::memcpy(k->image.data() + code_words, k->prog.pool.data(), k->prog.pool.size() * 4);
    void *dp = nullptr;
    cudaError_t e = ctx_alloc(c, &dp, k->image.size() * 4 + 16, k->pooled);
    k->d_code = static_cast<XInsn *>(dp);
    // ordered on the context's stream before any launch that reads it:
    // through the pinned stage when it is large enough (asynchronous), else
    // from the contract's own copy
    if (e == cudaSuccess) {
      std::lock_guard<std::mutex> g(c->load_mu);
      const size_t words = (k->image.size() + 3) & ~size_t(3);  // 16-byte steps
      if (words <= c->stage_words) {
        if (c->stage_off + words > c->stage_words) {
          // leave this half (its copies complete at the event) and take the
          // other one once its own copies are done
          e = cudaEventRecord(c->stage_ev[c->stage_half], c->stream);
          c->stage_pending[c->stage_half] = e == cudaSuccess;
          c->stage_half ^= 1;
          c->stage_off = 0;
          if (e == cudaSuccess && c->stage_pending[c->stage_half]) e = cudaEventSynchronize(c->stage_ev[c->stage_half]);
          c->stage_pending[c->stage_half] = false;
        }
        if (e == cudaSuccess) {
          uint32_t *dst = c->h_stage + size_t(c->stage_half) * c->stage_words + c->stage_off;
          std::memcpy(dst, k->image.data(), k->image.size() * 4);
          e = cudaMemcpyAsync(k->d_code, dst, k->image.size() * 4, cudaMemcpyHostToDevice, c->stream);
          c->stage_off += words;
        }
      } else {
        e = cudaMemcpyAsync(k->d_code, k->image.data(), k->image.size() * 4, cudaMemcpyHostToDevice, c->stream);
      }
    }
    if (e != cudaSuccess) {
      ctx_free(c, k->d_code, k->pooled);
      delete k;
      return cuda_fail(e, "program upload");
    }
    k->ctx = c;
    ++c->live_objects;
    *out = k;
    return PC_OK;
  } catch (const std::bad_alloc &) {
    return fail(PC_ENOMEM, "host allocation");
  } catch (...) {
    return fail(PC_EINVAL, "unexpected error in pc_load_payoff");
  }
}

pc_status pc_contract_destroy(pc_contract *k) {
  if (!k) return fail(PC_EINVAL, "null contract");
  cudaSetDevice(k->ctx->device);
  ctx_free(k->ctx, k->d_code, k->pooled);  // after the stream's launches that read it
  --k->ctx->live_objects;
  delete k;
  return PC_OK;
}

pc_status pc_cut_payoff(const uint32_t *bytecode, size_t n_words, const double *consts, size_t n_consts,
                        uint32_t *out_words, size_t cap_words, size_t *n_out_words, double *out_consts,
                        size_t cap_consts, size_t *n_out_consts) {
  if (!bytecode || !n_out_words || !n_out_consts || (n_consts && !consts)) return fail(PC_EINVAL, "null argument");
  if (n_words > PC_MAX_PROGRAM) return fail(PC_ELIMIT, "program exceeds PC_MAX_PROGRAM words");
  try {
    std::vector<uint32_t> w;
    std::vector<double> k;
    std::string e;
    pc_status s = cut_payoff(bytecode, n_words, consts, n_consts, w, k, e);
    if (s != PC_OK) return fail(s, e);
    *n_out_words = w.size();
    *n_out_consts = k.size();
    if (w.size() > cap_words || k.size() > cap_consts || (w.size() && !out_words) || (k.size() && !out_consts))
      return fail(PC_ELIMIT, "output buffers too small");
    std::copy(w.begin(), w.end(), out_words);
    std::copy(k.begin(), k.end(), out_consts);
    return PC_OK;
  } catch (const std::bad_alloc &) {
    return fail(PC_ENOMEM, "host allocation");
  }
}

pc_status pc_assemble(const char *text, uint32_t *words, size_t cap_words, size_t *n_words,
                      double *consts, size_t cap_consts, size_t *n_consts, char *err,
                      size_t err_cap) {
  if (!text || !n_words || !n_consts) return fail(PC_EINVAL, "null argument");
  try {
    std::vector<uint32_t> w;
    std::vector<double> k;
    std::string e;
    pc_status s = assemble_text(text, w, k, e);
    if (s != PC_OK) {
      if (err && err_cap) {
        std::strncpy(err, e.c_str(), err_cap - 1);
        err[err_cap - 1] = 0;
      }
      return fail(s, e);
    }
    *n_words = w.size();
    *n_consts = k.size();
    if (w.size() > cap_words || k.size() > cap_consts || (w.size() && !words) || (k.size() && !consts))
      return fail(PC_ELIMIT, "output buffers too small");
    std::copy(w.begin(), w.end(), words);
    std::copy(k.begin(), k.end(), consts);
    return PC_OK;
  } catch (const std::bad_alloc &) {
    return fail(PC_ENOMEM, "host allocation");
  }
}

pc_status pc_price_async(const pc_model *m, const pc_contract *k, uint64_t n_paths,
                         uint64_t path_offset, uint64_t seed, uint32_t stream, double *d_out) {
  if (!d_out) return fail(PC_EINVAL, "d_out is null");
  return run_price(m, k, n_paths, path_offset, seed, stream, d_out, nullptr);
}

pc_status pc_price_paths(const pc_model *m, const pc_contract *k, uint64_t n_paths,
                         uint64_t path_offset, uint64_t seed, uint32_t stream, double *d_out,
                         float *d_payoffs) {
  if (!d_out || !d_payoffs) return fail(PC_EINVAL, "null device output");
  return run_price(m, k, n_paths, path_offset, seed, stream, d_out, d_payoffs);
}

pc_status pc_price(const pc_model *m, const pc_contract *k, uint64_t n_paths, uint64_t seed,
                   double *out_price, double *out_stderr) {
  if (!out_price || !out_stderr) return fail(PC_EINVAL, "null output");
  if (n_paths < 2) return fail(PC_EINVAL, "n_paths must be >= 2 for a standard error");
  if (!m) return fail(PC_EINVAL, "null model");
  pc_ctx *c = m->ctx;
  pc_status s = run_price(m, k, n_paths, 0, seed, 0, c->d_res, nullptr);
  if (s != PC_OK) return s;
  // pinned read-back: the copy is queued and the bounded wait covers it
  CU(cudaMemcpyAsync(c->h_res, c->d_res, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "result copy");
  s = wait_stream(c);
  if (s != PC_OK) return s;
  double h[5];
  std::memcpy(h, c->h_res, sizeof(h));
  int32_t status;
  std::memcpy(&status, &h[4], 4);
  s = check_status(c, status);
  if (s != PC_OK) return s;
  const double n = double(n_paths), mean = h[0] / n;
  const double var = std::max(0.0, (h[1] - n * mean * mean) / (n - 1.0));
  *out_price = mean;
  *out_stderr = std::sqrt(var / n);
  return PC_OK;
}

pc_status pc_set_window_mode(pc_ctx *c, int32_t mode) {
  if (!c) return fail(PC_EINVAL, "null context");
  if (mode != PC_WINDOW_AUTO && mode != PC_WINDOW_SHARED && mode != PC_WINDOW_HBM)
    return fail(PC_EINVAL, "window mode must be PC_WINDOW_AUTO, _SHARED or _HBM");
  c->window_mode = mode;
  return PC_OK;
}

pc_status pc_debug_set_jit_pairs(pc_ctx *c, int32_t pairs) {
  if (!c) return fail(PC_EINVAL, "null context");
  if (pairs < 0 || pairs > 2) return fail(PC_EINVAL, "pairs must be 0 (automatic), 1 or 2");
  c->jit_pairs = pairs;
  return PC_OK;
}

pc_status pc_debug_set_cv_min_blocks(pc_ctx *c, int32_t blocks) {
  if (!c) return fail(PC_EINVAL, "null context");
  if (blocks < 0 || blocks > 16) return fail(PC_EINVAL, "blocks must be 0 (the kernel's default) .. 16");
  c->cv_min_blocks = blocks;
  return PC_OK;
}

pc_status pc_set_jit(pc_ctx *c, int32_t enabled) {
  if (!c) return fail(PC_EINVAL, "null context");
  if (enabled != 0 && enabled != 1) return fail(PC_EINVAL, "enabled must be 0 or 1");
  c->jit = enabled;
  return PC_OK;
}

pc_status pc_jit_compile(const pc_model *m, const pc_contract *k) {
  if (!m || !k) return fail(PC_EINVAL, "null model or contract");
  if (m->ctx != k->ctx) return fail(PC_EINVAL, "model and contract belong to different contexts");
  if (!jit_eligible(k)) return PC_OK;  // launches interpret it
  // the block a pricing launch of this pair uses (it does not depend on
  // the path count)
  Launch L;
  pc_status s = prepare(m, k, 1u << 20, 0, 0, 0, L, true);
  if (s != PC_OK) return s;
  CU(cudaSetDevice(m->ctx->device), "cudaSetDevice");
  cudaKernel_t jk = nullptr;
  const int wk = jit_window_kind(m->ctx, L);
  const size_t smem = jit_layout(m->ctx, k, L, wk);
  return jit_kernel(k, m->H.d, kJitPrice | wk, L.block, jk, jit_min_blocks(m->ctx, smem, L.block));
}

pc_status pc_price_info(const pc_model *m, const pc_contract *k, uint64_t n_paths, pc_launch_info *info) {
  if (!info) return fail(PC_EINVAL, "null info");
  Launch L;
  pc_status s = prepare(m, k, n_paths, 0, 0, 0, L, true);
  if (s != PC_OK) return s;
  const int d = m->H.d;
  info->window = L.args.lay.win;
  info->hbm_window = L.hbm_window ? 1 : 0;
  info->block = L.block;
  info->grid = L.grid;
  info->smem_bytes = L.smem;
  info->hbm_window_bytes =
      L.hbm_window ? uint64_t(L.grid) * L.block * uint64_t(L.args.lay.win) * d * sizeof(float2) : 0;
  info->window_bytes_written_per_path_date = L.hbm_window ? uint64_t(4 * d) : 0;
  return PC_OK;
}

pc_status pc_greeks(const pc_model *m, const pc_contract *k, uint64_t n_paths, uint64_t seed,
                    double *out_price, double *out_delta, double *out_vega, double *out_se) {
  if (!m || !k || !out_price || !out_delta || !out_vega || !out_se) return fail(PC_EINVAL, "null argument");
  if (n_paths < 2) return fail(PC_EINVAL, "n_paths must be >= 2 for a standard error");
  pc_ctx *c = m->ctx;
  const int d = m->H.d;
  for (int l = 0; l < d; ++l) {
    pc_status s = run_greeks(m, k, n_paths, 0, seed, l, c->d_gout + 8 * l, nullptr);
    if (s != PC_OK) return s;
  }
  double h[PC_MAX_UNDERLYINGS * 8], st[5];
  CU(cudaMemcpyAsync(h, c->d_gout, size_t(d) * 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
     "result copy");
  CU(cudaMemcpyAsync(st, c->d_res, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "status copy");
  pc_status s = wait_stream(c);
  if (s != PC_OK) return s;
  int32_t status;
  std::memcpy(&status, &st[4], 4);
  s = check_status(c, status);
  if (s != PC_OK) return s;
  const double n = double(n_paths);
  auto mean_se = [&](double sum, double sumsq, double &mean, double &se) {
    mean = sum / n;
    se = std::sqrt(std::max(0.0, (sumsq - n * mean * mean) / (n - 1.0)) / n);
  };
  mean_se(h[0], h[1], *out_price, out_se[0]);
  for (int l = 0; l < d; ++l) {
    mean_se(h[8 * l + 2], h[8 * l + 3], out_delta[l], out_se[1 + l]);
    mean_se(h[8 * l + 4], h[8 * l + 5], out_vega[l], out_se[1 + d + l]);
  }
  return PC_OK;
}

pc_status pc_debug_greeks_paths(const pc_model *m, const pc_contract *k, uint64_t n_paths,
                                uint64_t path_offset, uint64_t seed, int32_t underlying,
                                double *d_out, float *d_paths) {
  if (!m || !k || !d_out || !d_paths) return fail(PC_EINVAL, "null argument");
  if (underlying < 0 || underlying >= m->H.d) return fail(PC_EINVAL, "underlying out of range");
  return run_greeks(m, k, n_paths, path_offset, seed, underlying, d_out, d_paths);
}

pc_status pc_debug_philox(pc_ctx *c, const uint32_t *d_ctr, uint32_t key0, uint32_t key1,
                          uint32_t *d_out, size_t n) {
  if (!c || (n && (!d_ctr || !d_out))) return fail(PC_EINVAL, "null argument");
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  CU(launch_debug_philox(d_ctr, key0, key1, d_out, n, c->stream), "philox kernel");
  return wait_stream(c);
}

pc_status pc_debug_paths(const pc_model *m, uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                         uint32_t stream, float *d_S) {
  if (!m || !d_S) return fail(PC_EINVAL, "null argument");
  if (n_paths > (uint64_t(1) << 24)) return fail(PC_ELIMIT, "n_paths too large for the probe");
  Program empty;
  Layout lay = make_layout(empty, m->H, 1);
  lay.stack = 0;
  lay.off_bstack = 0;
  lay.off_cache = m->H.bstack * m->H.d;
  lay.off_win = lay.off_cache;
  lay.words = lay.off_win + m->H.d;
  pc_ctx *c = m->ctx;
  if (size_t(lay.words) * 32 * 8 + 2048 > size_t(c->max_smem)) return fail(PC_ELIMIT, "model too large for the probe");
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  CU(launch_debug_paths(m->dev, lay, n_paths, path_offset, uint32_t(seed), uint32_t(seed >> 32),
                        stream, d_S, c->stream),
     "paths kernel");
  return wait_stream(c);
}

pc_status pc_debug_program(const uint32_t *bytecode, size_t n_words, const double *consts,
                           size_t n_consts, const int32_t *template_params, size_t n_params,
                           int32_t p1, int32_t p2, uint32_t *out, size_t cap_words,
                           size_t *n_insn, size_t *n_pool) {
  if (!n_insn || !n_pool) return fail(PC_EINVAL, "null argument");
  try {
    Program p;
    std::string err;
    pc_status s = compile_program(bytecode, n_words, consts, n_consts, template_params, n_params,
                                  p1, p2, true, p, err);
    if (s != PC_OK) return fail(s, err);
    *n_insn = p.code.size();
    *n_pool = p.pool.size();
    if (4 * p.code.size() + p.pool.size() > cap_words || !out)
      return fail(PC_ELIMIT, "output buffer too small");
    std::memcpy(out, p.code.data(), p.code.size() * sizeof(XInsn));
    std::memcpy(out + 4 * p.code.size(), p.pool.data(), p.pool.size() * sizeof(float));
    return PC_OK;
  } catch (const std::bad_alloc &) {
    return fail(PC_ENOMEM, "host allocation");
  }
}

pc_status pc_debug_bridge(const pc_model_desc *desc, int32_t *date_ops, uint32_t *ops,
                          size_t cap_ops, size_t *n_ops) {
  if (!desc || !n_ops) return fail(PC_EINVAL, "null argument");
  ModelHost H;
  std::string err;
  pc_status s = build_model(*desc, H, err);
  if (s != PC_OK) return fail(s, err);
  *n_ops = H.ops.size();
  if (H.ops.size() > cap_ops || !ops || !date_ops) return fail(PC_ELIMIT, "output buffer too small");
  std::copy(H.date_ops.begin(), H.date_ops.end(), date_ops);
  for (size_t i = 0; i < H.ops.size(); ++i) {
    const BridgeOp &o = H.ops[i];
    uint32_t *w = ops + 6 * i;
    std::memcpy(w + 0, &o.wl, 4);
    std::memcpy(w + 1, &o.wr, 4);
    std::memcpy(w + 2, &o.sd, 4);
    w[3] = o.j;
    w[4] = uint32_t(o.flags) << 16;
    w[5] = o.m;
  }
  return PC_OK;
}

}  // extern "C"
