// pc_kernels.cu -- device side of the payoff-expression Monte Carlo engine.
//
// One fused kernel keeps each path on chip from random numbers to payoff:
//   Philox4x32-10 (Salmon et al., SC'11) -> 24-bit uniforms -> Box-Muller
//   -> Brownian bridge (breadth-first bisection, produced lazily in date
//   order) -> X = L W -> GBM S_l = S0_l 2^(A_l(o) + sum_k B_lk W_k)
//   -> the payoff expression (IL of Sec. 3, semantics of Fig. 3) run by a
//   warp-uniform stack machine -> per-tile FP64 sums.
// No path value is written to global memory.  Per-thread state (operand
// stack, loop frames, bridge stack, per-level Philox block caches, the
// window of recent dates) lives in shared memory as word-interleaved slots:
// word w of thread t is at region[w * kBlock + t], so the warp-uniform slot
// indices of the interpreter give conflict-free accesses.
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "pc_device.cuh"
#include "pc_internal.h"
#include "pc_eval.cuh"
#include "pc_price.cuh"

namespace pc {

namespace {


// Tiles of kTilePaths consecutive paths (two per lane: tile*64 + lane and
// tile*64 + 32 + lane) are handed to warps through an atomic counter
// (price_tiles, pc_price.cuh).  GW: the window of simulated dates lives in
// HBM (lay.gwin) instead of shared memory, for programs that look back
// further than shared memory holds.
template <int D, bool WRITE, bool GW = false>
__global__ void __launch_bounds__(kBlock) price_kernel(const __grid_constant__ PriceArgs a) {
  price_tiles<D, WRITE>(a, [&](const uint4 *P, const float *pool, float2 *R, const Rng2 &g, bool live0,
                               bool live1, const float(&Bm)[D * D], const float(&S0)[D]) {
    return eval_path<D, GW>(P, pool, R, a, g, live0, live1, Bm, S0);
  });
}

// Portfolio kernels.  Warps take work units (a contract and a run of its
// tiles) from the launch's counter in the order of the unit array.  When a
// warp's unit belongs to another contract than its previous one, the warp
// copies that contract's arguments into its own slot of shared memory; the
// program and constant pool are read from global memory through L1.  The
// tiles run as in price_kernel and finish into the contract's own reduction
// scratch, so each contract's sums are those of a single-contract launch.
// batch_kernel<d> serves the contracts of one underlying count;
// batch_kernel_any serves every count in one launch (the unit's contract
// selects the generator), at the register bound the four-underlying
// generator needs.

// The tiles of unit U of contract a (arguments in the warp's slot).
template <int D>
__device__ __forceinline__ void batch_unit(const PriceArgs &a, const BatchUnit &U, float2 *R, int lane) {
  const uint4 *P = reinterpret_cast<const uint4 *>(a.prog);
  const float *pool = reinterpret_cast<const float *>(P + a.n_insn);
  float Bm[D * D], S0[D];
  load_model_regs<D>(a.m, Bm, S0);
  Rng2 g;
  g.stream = a.stream;
#pragma unroll
  for (int i = 0; i < 20; ++i) g.rk[i] = a.rk[i];
  for (uint32_t k = 0; k < U.n_tiles; ++k) {
    const uint64_t tile = U.tile0 + k;
    const uint64_t i0 = tile * kTilePaths + lane, i1 = i0 + 32;
    const bool live0 = i0 < a.n_paths, live1 = i1 < a.n_paths;
    const uint64_t p0 = a.path_offset + i0, p1 = a.path_offset + i1;
    g.plo[0] = uint32_t(p0);
    g.phi[0] = uint32_t(p0 >> 32);
    g.plo[1] = uint32_t(p1);
    g.phi[1] = uint32_t(p1 >> 32);
    const float2 x = eval_path<D>(P, pool, R, a, g, live0, live1, Bm, S0);
    Moments<2> mo;
    if (live0) {
      mo.add(0, x.x);
      mo.add_prod(1, x.x, x.x);
    }
    if (live1) {
      mo.add(0, x.y);
      mo.add_prod(1, x.y, x.y);
    }
    double tp[2];
    mo.warp_total(tp);
    finish_tile<2>(a, tile, tp, lane);
  }
}

// The unit loop; RUN(a, U, R, lane) runs one unit.
template <typename RUN>
__device__ __forceinline__ void batch_units(const BatchArgs &b, RUN run) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *slot = smem + (b.slot_bytes / 4) * warp;
  float2 *R = reinterpret_cast<float2 *>(smem + (b.slot_bytes / 4) * (blockDim.x >> 5)) + threadIdx.x;
  const PriceArgs &a = *reinterpret_cast<const PriceArgs *>(slot);
  uint32_t cur = 0xffffffffu;
  for (;;) {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd(b.counter, 1ull);
    u = __shfl_sync(kFull, u, 0);
    if (u >= b.n_units) break;
    const BatchUnit U = b.units[u];
    if (U.item != cur) {
      __syncwarp();
      const uint32_t *src = reinterpret_cast<const uint32_t *>(b.items + U.item);
      for (int i = lane; i < int(sizeof(PriceArgs) / 4); i += 32) slot[i] = __ldg(src + i);
      __syncwarp();
      cur = U.item;
    }
    run(a, U, R, lane);
  }
}

// At least 5 resident 128-thread blocks (<= 102 registers): -4 % per
// portfolio replay against the uncapped 112 registers, 6 blocks spill.
template <int D>
__global__ void __launch_bounds__(kBlock, 5) batch_kernel(const BatchArgs b) {
  batch_units(b, [](const PriceArgs &a, const BatchUnit &U, float2 *R, int lane) { batch_unit<D>(a, U, R, lane); });
}

__global__ void __launch_bounds__(kBlock, 5) batch_kernel_any(const BatchArgs b) {
  batch_units(b, [](const PriceArgs &a, const BatchUnit &U, float2 *R, int lane) {
    switch (a.m.d) {
      case 1: batch_unit<1>(a, U, R, lane); break;
      case 2: batch_unit<2>(a, U, R, lane); break;
      case 3: batch_unit<3>(a, U, R, lane); break;
      default: batch_unit<4>(a, U, R, lane); break;
    }
  });
}

__global__ void debug_philox_kernel(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                    size_t n) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = reinterpret_cast<const uint4 *>(ctr)[i];
  reinterpret_cast<uint4 *>(out)[i] = philox(c, k0, k1);
}

// Thread t generates paths offset + 2t and offset + 2t + 1 with the pricing
// kernel's generator and writes every date of both.
template <int D>
__global__ void __launch_bounds__(kBlock) debug_paths_kernel(const __grid_constant__ ModelDev m, const Layout lay,
                                                             uint64_t n_paths, uint64_t offset,
                                                             const __grid_constant__ RoundKeys rk,
                                                             uint32_t stream, float *out) {
  extern __shared__ __align__(16) uint32_t smem[];
  float2 *R = reinterpret_cast<float2 *>(smem) + threadIdx.x;
  const uint64_t i0 = 2 * (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x), i1 = i0 + 1;
  if (i0 >= n_paths) return;
  float Bm[D * D], S0[D];
  load_model_regs<D>(m, Bm, S0);
  Rng2 g;
  g.plo[0] = uint32_t(offset + i0);
  g.phi[0] = uint32_t((offset + i0) >> 32);
  g.plo[1] = uint32_t(offset + i1);
  g.phi[1] = uint32_t((offset + i1) >> 32);
  g.stream = stream;
#pragma unroll
  for (int i = 0; i < 20; ++i) g.rk[i] = rk.k[i];
  PathState<D> ps;
  path_state_init<D>(ps, R, lay);
  const size_t row = size_t(m.n) + 1;
  const bool has1 = i1 < n_paths;
  for (int l = 0; l < D; ++l) {
    out[(i0 * D + l) * row] = S0[l];
    if (has1) out[(i1 * D + l) * row] = S0[l];
  }
  for (int t = 1; t <= m.n; ++t) {
    gen_date<D>(t, ps, m, lay, g, R, Bm, S0);
    const int ws = lay.off_win + (t & (lay.win - 1)) * D;
    for (int l = 0; l < D; ++l) {
      const float2 v = SL(ws + l);
      out[(i0 * D + l) * row + t] = v.x;
      if (has1) out[(i1 * D + l) * row + t] = v.y;
    }
  }
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

}  // namespace

cudaError_t launch_price(const PriceArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
  const bool w = a.out_paths != nullptr, gw = a.lay.gwin != nullptr;
#define LAUNCH(DD, WW, GG)                                                         \
  do {                                                                             \
    auto k = price_kernel<DD, WW, GG>;                                             \
    cudaError_t e = set_smem(k, smem);                                             \
    if (e != cudaSuccess) return e;                                                \
    k<<<grid, block, smem, s>>>(a);                                                \
    return cudaGetLastError();                                                     \
  } while (0)
#define LAUNCH_D(DD)                                                               \
  do {                                                                             \
    if (gw) { if (w) LAUNCH(DD, true, true); else LAUNCH(DD, false, true); }       \
    else { if (w) LAUNCH(DD, true, false); else LAUNCH(DD, false, false); }        \
  } while (0)
  switch (a.m.d) {
    case 1: LAUNCH_D(1);
    case 2: LAUNCH_D(2);
    case 3: LAUNCH_D(3);
    case 4: LAUNCH_D(4);
    default: return cudaErrorInvalidValue;
  }
#undef LAUNCH_D
#undef LAUNCH
}

namespace {
int price_occupancy(uint64_t v, int block, size_t smem) {
  const int d = int(v & 0xff);
  const bool hbm_window = (v >> 8) & 1;
  int nb = 0;
  cudaError_t e = cudaSuccess;
#define OCC(DD)                                                                                      \
  do {                                                                                               \
    if (hbm_window) {                                                                                \
      set_smem(price_kernel<DD, false, true>, smem);                                                 \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<DD, false, true>, block, smem); \
    } else {                                                                                         \
      set_smem(price_kernel<DD, false, false>, smem);                                                \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<DD, false, false>, block, smem); \
    }                                                                                                \
  } while (0)
  switch (d) {
    case 0:
      e = set_smem(batch_kernel_any, smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel_any, block, smem);
      break;
    case 1: OCC(1); break;
    case 2: OCC(2); break;
    case 3: OCC(3); break;
    case 4: OCC(4); break;
    default: return 0;
  }
#undef OCC
  return e == cudaSuccess ? nb : 0;
}
}  // namespace

int price_blocks_per_sm(int d, int block, size_t smem, bool hbm_window, bool memoise) {
  return occupancy_memo((uint64_t(1) << 32) | (uint64_t(hbm_window) << 8) | uint64_t(d), block, smem,
                        price_occupancy, memoise);
}

int occupancy_memo(uint64_t variant, int block, size_t smem, int (*query)(uint64_t, int, size_t),
                   bool store) {
  static std::mutex mu;
  static std::map<std::tuple<int, uint64_t, int, size_t>, int> memo;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return query(variant, block, smem);
  const auto key = std::make_tuple(dev, variant, block, smem);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
  }
  const int nb = query(variant, block, smem);
  if (nb > 0 && store) {
    std::lock_guard<std::mutex> g(mu);
    memo[key] = nb;
  }
  return nb;
}

int batch_blocks_per_sm(int d, int block, size_t smem) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define OCC(DD)                                                                     \
  do {                                                                              \
    e = set_smem(batch_kernel<DD>, smem);                                           \
    if (e == cudaSuccess)                                                           \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<DD>, block, smem); \
  } while (0)
  switch (d) {
    case 0:
      e = set_smem(batch_kernel_any, smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel_any, block, smem);
      break;
    case 1: OCC(1); break;
    case 2: OCC(2); break;
    case 3: OCC(3); break;
    case 4: OCC(4); break;
    default: return 0;
  }
#undef OCC
  return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_batch(const BatchArgs &b, int d, int grid, int block, size_t smem, cudaStream_t s) {
  switch (d) {
    case 0: batch_kernel_any<<<grid, block, smem, s>>>(b); break;
    case 1: batch_kernel<1><<<grid, block, smem, s>>>(b); break;
    case 2: batch_kernel<2><<<grid, block, smem, s>>>(b); break;
    case 3: batch_kernel<3><<<grid, block, smem, s>>>(b); break;
    case 4: batch_kernel<4><<<grid, block, smem, s>>>(b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int max_dynamic_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v;
}

cudaError_t launch_debug_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  debug_philox_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(ctr, k0, k1, out, n);
  return cudaGetLastError();
}

cudaError_t launch_debug_paths(const ModelDev &m, const Layout &lay, uint64_t n_paths,
                               uint64_t offset, uint32_t k0, uint32_t k1, uint32_t stream,
                               float *out, cudaStream_t s) {
  int block = kBlock;
  while (block > 32 && size_t(lay.words) * block * 8 + 2048 > size_t(max_dynamic_smem())) block /= 2;
  const size_t smem = size_t(lay.words) * block * 8;
  const unsigned grid = unsigned((n_paths + 2 * block - 1) / (2 * block));
  RoundKeys rk;
  philox_round_keys(uint64_t(k0) | (uint64_t(k1) << 32), rk.k);
  if (grid == 0) return cudaSuccess;
#define DLAUNCH(DD)                                                                 \
  do {                                                                              \
    auto k = debug_paths_kernel<DD>;                                                \
    cudaError_t e = set_smem(k, smem);                                              \
    if (e != cudaSuccess) return e;                                                 \
    k<<<grid, block, smem, s>>>(m, lay, n_paths, offset, rk, stream, out);          \
    return cudaGetLastError();                                                      \
  } while (0)
  switch (m.d) {
    case 1: DLAUNCH(1);
    case 2: DLAUNCH(2);
    case 3: DLAUNCH(3);
    case 4: DLAUNCH(4);
    default: return cudaErrorInvalidValue;
  }
#undef DLAUNCH
}

// Scratch of pc_price_noalloc: the reduction control block (counters and
// chunk partials, kControlBytes) first, then one (sum, sum of squares) pair
// per tile of kTilePaths paths for up to PC_NOALLOC_MAX_PATHS paths.
// Zero-initialised when the module loads; each call clears the control
// block again before its launch.
constexpr size_t kNoAllocScratchBytes =
    kNoAllocCounterBytes + (PC_NOALLOC_MAX_PATHS / kTilePaths) * 2 * sizeof(double);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

cudaError_t noalloc_scratch(void **ptr, size_t *bytes) {
  constexpr int kMaxDevices = 64;
  static void *addr[kMaxDevices] = {};
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *ptr = addr[dev];
  *bytes = kNoAllocScratchBytes;
  return cudaSuccess;
}


}  // namespace pc
