// pc_price.cuh -- the pricing kernel's body: program staging, the tile
// loop and the per-tile reduction, generic in the payoff evaluator
// (the interpreter eval_path, or a run-time specialised evaluator).
#pragma once

#include "pc_device.cuh"

namespace pc {

// EVAL(P, pool, R, g, live0, live1, Bm, S0) -> float2 payoffs of the lane's
// two paths.
template <int D, bool WRITE, typename EVAL>
__device__ __forceinline__ void price_tiles(const PriceArgs &a, EVAL eval) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int last_block;
  uint4 *P = reinterpret_cast<uint4 *>(smem);
  const int prog_words = a.n_insn * 4 + a.n_pool;
  const uint32_t *src = reinterpret_cast<const uint32_t *>(a.prog);
  for (int i = threadIdx.x; i < prog_words; i += blockDim.x) smem[i] = src[i];
  __syncthreads();
  const float *pool = reinterpret_cast<const float *>(smem + a.n_insn * 4);
  float2 *R = reinterpret_cast<float2 *>(smem + prog_words) + threadIdx.x;
  const float(&Bm)[D * D] = *reinterpret_cast<const float(*)[D * D]>(a.m.Bv);
  const float(&S0)[D] = *reinterpret_cast<const float(*)[D]>(a.m.S0v);
  const int lane = threadIdx.x & 31;
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.control);
  Rng2 g;
  g.stream = a.stream;
#pragma unroll
  for (int i = 0; i < 20; ++i) g.rk[i] = a.rk[i];
  for (;;) {
    unsigned long long tile = 0;
    if (lane == 0) tile = atomicAdd(ctr, 1ull);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= a.n_tiles) break;
    const uint64_t i0 = tile * kTilePaths + lane, i1 = i0 + 32;
    const bool live0 = i0 < a.n_paths, live1 = i1 < a.n_paths;
    const uint64_t p0 = a.path_offset + i0, p1 = a.path_offset + i1;
    g.plo[0] = uint32_t(p0);
    g.phi[0] = uint32_t(p0 >> 32);
    g.plo[1] = uint32_t(p1);
    g.phi[1] = uint32_t(p1 >> 32);
    const float2 x = eval(P, pool, R, g, live0, live1, Bm, S0);
    Moments<2> mo;
    if (live0) {
      mo.add(0, x.x);
      mo.add_prod(1, x.x, x.x);
      if (WRITE) a.out_paths[i0] = x.x;
    }
    if (live1) {
      mo.add(0, x.y);
      mo.add_prod(1, x.y, x.y);
      if (WRITE) a.out_paths[i1] = x.y;
    }
    double tp[2];
    mo.warp_total(tp);
    finish_tile<2>(a, tile, tp, lane);
  }
  // the last block to exit re-zeroes the tile counter: no warp grabs tiles
  // any more once every block has left its loop
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_block = atomicAdd(ctr + 1, 1ull) == gridDim.x - 1;
  }
  __syncthreads();
  if (last_block && threadIdx.x == 0) {
    ctr[0] = 0;
    ctr[1] = 0;
  }
}

#if PC_PAIRS == 2
// The same with four paths a lane (two pairs): warps take pairs of
// consecutive tiles (2u, 2u + 1) from the counter; pair h of the lane holds
// tile 2u + h's paths lane and lane + 32, exactly as a one-pair lane holds a
// tile, so every path's value and every tile's partials are those of
// price_tiles.  EVAL(P, pool, R, g, live, Bm, S0) -> PV of the lane's four
// paths.
template <int D, bool WRITE, typename EVAL>
__device__ __forceinline__ void price_tiles2(const PriceArgs &a, EVAL eval) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int last_block;
  uint4 *P = reinterpret_cast<uint4 *>(smem);
  const int prog_words = a.n_insn * 4 + a.n_pool;
  const uint32_t *src = reinterpret_cast<const uint32_t *>(a.prog);
  for (int i = threadIdx.x; i < prog_words; i += blockDim.x) smem[i] = src[i];
  __syncthreads();
  const float *pool = reinterpret_cast<const float *>(smem + a.n_insn * 4);
  float2 *R = reinterpret_cast<float2 *>(smem + prog_words) + threadIdx.x;
  const float(&Bm)[D * D] = *reinterpret_cast<const float(*)[D * D]>(a.m.Bv);
  const float(&S0)[D] = *reinterpret_cast<const float(*)[D]>(a.m.S0v);
  const int lane = threadIdx.x & 31;
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.control);
  const uint64_t n_pairs = (a.n_tiles + 1) / 2;
  RngH<2> g;
  g.stream = a.stream;
#pragma unroll
  for (int i = 0; i < 20; ++i) g.rk[i] = a.rk[i];
  for (;;) {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd(ctr, 1ull);
    u = __shfl_sync(kFull, u, 0);
    if (u >= n_pairs) break;
    uint64_t idx[4];
    bool live[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      idx[q] = (2 * u + (q >> 1)) * kTilePaths + lane + 32 * (q & 1);
      live[q] = idx[q] < a.n_paths;
      const uint64_t pq = a.path_offset + idx[q];
      g.plo[q] = uint32_t(pq);
      g.phi[q] = uint32_t(pq >> 32);
    }
    const PV x = eval(P, pool, R, g, live, Bm, S0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t tile = 2 * u + h;
      if (tile >= a.n_tiles) break;  // warp-uniform
      const float x0 = pv_get(x, 2 * h), x1 = pv_get(x, 2 * h + 1);
      Moments<2> mo;
      if (live[2 * h]) {
        mo.add(0, x0);
        mo.add_prod(1, x0, x0);
        if (WRITE) a.out_paths[idx[2 * h]] = x0;
      }
      if (live[2 * h + 1]) {
        mo.add(0, x1);
        mo.add_prod(1, x1, x1);
        if (WRITE) a.out_paths[idx[2 * h + 1]] = x1;
      }
      double tp[2];
      mo.warp_total(tp);
      finish_tile<2>(a, tile, tp, lane);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_block = atomicAdd(ctr + 1, 1ull) == gridDim.x - 1;
  }
  __syncthreads();
  if (last_block && threadIdx.x == 0) {
    ctr[0] = 0;
    ctr[1] = 0;
  }
}
#endif

}  // namespace pc
