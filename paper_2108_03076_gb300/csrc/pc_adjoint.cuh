// pc_adjoint.cuh -- pathwise delta and vega of every underlying in one
// launch, by the chain rule in reverse (adjoint mode).
//
// Forward sweep: the payoff program runs as in the pricing interpreter (two
// paths per lane, the warp in step) and records a tape of the real-valued
// arithmetic the path's result is computed from.  Every real value carries
// the number of the tape entry that produced it (-1 for constants: literals,
// discounts, history); an operation whose inputs carry entries appends one
// entry: the numbers of its (at most two) inputs, which are the same in
// every lane because the warp runs one instruction stream, and each lane's
// partial derivatives with respect to them -- decisions held fixed: min,
// max, if and a loop's latch pass the derivative to the operand each path
// chose.  A model read of label l at ordinal o >= 0 is a leaf entry holding
// the path state of that date that the parameters act on: under the GBM
// solution S_l(o) = S0_l exp((r - sigma_l^2 / 2) tau_o + sigma_l X_l(o)),
// with X = L W independent of the parameters, dS/dS0_l = S / S0_l and
// dS/dsigma_l = S (X_l(o) - sigma_l tau_o) (a per-date checkpoint of S and
// X; ordinal 0 gives 1 and 0).  So the reverse sweep needs no path values
// and no re-simulation.
//
// Reverse sweep: the adjoint of the result is 1; entries are visited from
// the last to the first, each adding its adjoint times its partials into
// its inputs' adjoints, and a leaf into the delta and vega accumulators of
// its label.  All d deltas and d vegas of the path come out of one sweep,
// whatever d.
//
// The tape lives in HBM, one region per resident warp (TapeArgs), reused
// tile after tile: entry e of lane l at [e * 32 + l] (coalesced for the
// warp's common entry number).  Its capacity is the load-time bound on the
// entries a run of the program can append (pc_adjoint_api.cpp); an overflow
// raises the status word and stops recording.
#pragma once

#include "pc_device.cuh"

namespace pc {

namespace {

__device__ __forceinline__ float2 adsel(float2 c, float2 p, float2 q) {
  return make_float2(bits(c.x) ? p.x : q.x, bits(c.y) ? p.y : q.y);
}

// The adjoint launch's per-warp tape cursor and recording.
struct Tape {
  float4 *part;
  float2 *adj;
  int2 *ids;
  int emax, n, lane;
  int32_t *status;
  // Append an entry with inputs (i1, i2) and partials (p1, p2); the result's
  // entry number, or -1 when no input carries one (a constant result).
  __device__ __forceinline__ int add(int i1, int i2, float2 p1, float2 p2) {
    if (i1 < 0 && i2 < 0) return -1;
    return put(i1, i2, i1 < 0 ? make_float2(0.f, 0.f) : p1, i2 < 0 ? make_float2(0.f, 0.f) : p2);
  }
  __device__ __forceinline__ int put(int i1, int i2, float2 p1, float2 p2) {
    if (n >= emax) {  // beyond the load-time bound: report, stop recording
      if (lane == 0) atomicOr(status, 4);
      return -1;
    }
    const int e = n++;
    part[size_t(e) * 32 + lane] = make_float4(p1.x, p1.y, p2.x, p2.y);
    adj[size_t(e) * 32 + lane] = make_float2(0.f, 0.f);
    if (lane == 0) ids[e] = make_int2(i1, i2);
    return e;
  }
};

// Leaf of label l at ordinal o (read value s): the GBM partials, or none
// for a constant (history).
template <int D>
__device__ __forceinline__ int adj_leaf(Tape &T, int o, int l, float2 s, float scale, const float2 *R,
                                        const ModelDev &m, const Layout &lay, const float (&S0)[D]) {
  if (o < 0) return -1;
  if (o == 0) return T.put(-2 - l, -1, make_float2(scale, scale), make_float2(0.f, 0.f));
  const float2 x = SL(lay.off_xwin + (o & (lay.win - 1)) * D + l);
  const float st = __fmul_rn(__ldg(m.sig + l), __ldg(m.tau + o));
  const float r0 = __fdiv_rn(scale, S0[l]);
  return T.put(-2 - l, -1, make_float2(__fmul_rn(s.x, r0), __fmul_rn(s.y, r0)),
               make_float2(__fmul_rn(__fmul_rn(s.x, __fsub_rn(x.x, st)), scale),
                           __fmul_rn(__fmul_rn(s.y, __fsub_rn(x.y, st)), scale)));
}

// The payoff program of two paths per lane with its tape (forward sweep);
// returns the result and sets `res` to its entry number.
template <int D>
__device__ float2 eval_adjoint(const uint4 *P, const float *pool, float2 *R, const PriceArgs &a,
                               const Rng2 &g, bool live0, bool live1, const float (&Bm)[D * D],
                               const float (&S0)[D], const float (&Lm)[D * D], Tape &T, int &res) {
#include "pc_adjoint_state.inc"
  for (;;) {
    const uint4 I = P[pc];
    const uint32_t op = I.x & 0xffu;
    const float kk = __uint_as_float(I.y);
#include "pc_adjoint_ops.inc"
  }
}

// Reverse sweep of one tile's tape: the per-path derivatives of the result
// with respect to S0_l (dS) and sigma_l (dv).
template <int D>
__device__ __forceinline__ void reverse_sweep(Tape &T, int res, float2 (&dS)[D], float2 (&dv)[D]) {
#pragma unroll
  for (int l = 0; l < D; ++l) dS[l] = dv[l] = make_float2(0.f, 0.f);
  if (res < 0) return;
  const int lane = T.lane;
  T.adj[size_t(res) * 32 + lane] = make_float2(1.f, 1.f);
  for (int e = T.n - 1; e >= 0; --e) {
    const float2 ad = T.adj[size_t(e) * 32 + lane];
    const int2 in = T.ids[e];
    const float4 p = T.part[size_t(e) * 32 + lane];
    if (in.x <= -2) {
      const int l = -2 - in.x;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        if (q == l) {
          dS[q] = make_float2(__fmaf_rn(ad.x, p.x, dS[q].x), __fmaf_rn(ad.y, p.y, dS[q].y));
          dv[q] = make_float2(__fmaf_rn(ad.x, p.z, dv[q].x), __fmaf_rn(ad.y, p.w, dv[q].y));
        }
      }
      continue;
    }
    if (in.x >= 0) {
      float2 &t = T.adj[size_t(in.x) * 32 + lane];
      t = make_float2(__fmaf_rn(ad.x, p.x, t.x), __fmaf_rn(ad.y, p.y, t.y));
    }
    if (in.y >= 0) {
      float2 &t = T.adj[size_t(in.y) * 32 + lane];
      t = make_float2(__fmaf_rn(ad.x, p.z, t.x), __fmaf_rn(ad.y, p.w, t.y));
    }
  }
}

}  // namespace

// The sensitivity launch: per path (x, dx/dS0_l, dx/dsigma_l for l < D), per
// tile the FP64 sums and sums of squares of the 1 + 2D values in the
// deterministic chunked reduction (width 2 (1 + 2D)).
// EVAL(P, pool, R, g, live0, live1, Bm, S0, Lm, T, res) -> the lane's two
// payoffs with the tape (eval_adjoint, or a run-time specialised evaluator).
template <int D, bool WRITE, typename EVAL>
__device__ __forceinline__ void adjoint_tiles(const PriceArgs &a, const TapeArgs &ta, EVAL eval) {
  constexpr int V = 1 + 2 * D, W = 2 * V;
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
  float Lm[D * D];
#pragma unroll
  for (int i = 0; i < D * D; ++i) Lm[i] = __ldg(a.m.L + i);
  const int lane = threadIdx.x & 31;
  const size_t gw = size_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  Tape T;
  T.part = ta.part + gw * size_t(ta.emax) * 32;
  T.adj = ta.adj + gw * size_t(ta.emax) * 32;
  T.ids = ta.ids + gw * size_t(ta.emax);
  T.emax = ta.emax;
  T.lane = lane;
  T.status = a.status;
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
    T.n = 0;
    int res = -1;
    const float2 x = eval(P, pool, R, g, live0, live1, Bm, S0, Lm, T, res);
    __syncwarp();  // the ids lane 0 wrote are read by every lane
    float2 dS[D], dv[D];
    reverse_sweep<D>(T, res, dS, dv);
    __syncwarp();  // the next tile reuses the region
    float q0[V], q1[V];
    q0[0] = x.x;
    q1[0] = x.y;
#pragma unroll
    for (int l = 0; l < D; ++l) {
      q0[1 + l] = dS[l].x;
      q1[1 + l] = dS[l].y;
      q0[1 + D + l] = dv[l].x;
      q1[1 + D + l] = dv[l].y;
    }
    Moments<W> mo;
    if (live0) {
#pragma unroll
      for (int j = 0; j < V; ++j) {
        mo.add(2 * j, q0[j]);
        mo.add_prod(2 * j + 1, q0[j], q0[j]);
        if (WRITE) a.out_paths[i0 * V + j] = q0[j];
      }
    }
    if (live1) {
#pragma unroll
      for (int j = 0; j < V; ++j) {
        mo.add(2 * j, q1[j]);
        mo.add_prod(2 * j + 1, q1[j], q1[j]);
        if (WRITE) a.out_paths[i1 * V + j] = q1[j];
      }
    }
    double tp[W];
    mo.warp_total(tp);
    finish_tile<W>(a, tile, tp, lane);
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

}  // namespace pc
