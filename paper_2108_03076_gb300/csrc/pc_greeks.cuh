// pc_greeks.cuh -- pathwise sensitivities of the Monte Carlo price.
//
// For one underlying g per launch, every value of the payoff program carries
// two tangents next to it: d/dS0_g and d/dsigma_g of the path's payoff,
// holding every discrete decision (if, loopif, comparisons) fixed -- the
// pathwise derivative, valid for payoffs that are Lipschitz in the path.
// Tangents enter at the model reads: under the GBM
//   S_g(o) = S0_g exp((r - sigma_g^2 / 2) tau_o + sigma_g X_g(o)),  X = L W,
// dS_g(o)/dS0_g = S_g(o) / S0_g and dS_g(o)/dsigma_g = S_g(o) (X_g(o) -
// sigma_g tau_o); every other read has zero tangents.  Arithmetic
// propagates them by the chain rule (forward / tangent mode).  The paths,
// random numbers and program are exactly those of the pricing kernel, so
// the price and both sensitivities come from common random numbers.
//
// Each logical stack slot s of the program occupies three physical slots
// 3s (value), 3s + 1 (d/dS0), 3s + 2 (d/dsigma); loop frames likewise.
//
// The tangent evaluator is shared by the interpreting kernel (eval_greeks)
// and the run-time specialised one: its state is pc_greeks_state.inc and
// its instruction cases pc_greeks_ops.inc.
#pragma once

#include "pc_device.cuh"

namespace pc {

struct TV {
  float2 v, a, b;  // value, d/dS0_g, d/dsigma_g (two paths each)
};

__device__ __forceinline__ TV tv(float2 v) { return {v, make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
// Every real operation rounds on its own (explicit _rn intrinsics, products
// accumulated by explicit FMAs), so the specialised evaluator, which sees
// across instruction boundaries, contracts nothing the interpreter does not.
__device__ __forceinline__ float2 add2(float2 p, float2 q) { return f2(__fadd_rn(p.x, q.x), __fadd_rn(p.y, q.y)); }
__device__ __forceinline__ float2 sub2(float2 p, float2 q) { return f2(__fsub_rn(p.x, q.x), __fsub_rn(p.y, q.y)); }
__device__ __forceinline__ float2 mul2(float2 p, float2 q) { return f2(__fmul_rn(p.x, q.x), __fmul_rn(p.y, q.y)); }
// p q + r per lane with one rounding
__device__ __forceinline__ float2 fma2(float2 p, float2 q, float2 r) {
  return f2(__fmaf_rn(p.x, q.x, r.x), __fmaf_rn(p.y, q.y, r.y));
}
__device__ __forceinline__ float2 scl2(float2 p, float k) { return f2(__fmul_rn(p.x, k), __fmul_rn(p.y, k)); }
__device__ __forceinline__ float2 neg2(float2 p) { return f2(-p.x, -p.y); }
__device__ __forceinline__ float2 sel2(float2 c, float2 p, float2 q) {
  return f2(bits(c.x) ? p.x : q.x, bits(c.y) ? p.y : q.y);
}

// Slot access of the value-with-tangents stack.
__device__ __forceinline__ TV ldv(float2 *R, int s) { return {SL(3 * s), SL(3 * s + 1), SL(3 * s + 2)}; }
__device__ __forceinline__ void stv(float2 *R, int s, const TV &x) {
  SL(3 * s) = x.v;
  SL(3 * s + 1) = x.a;
  SL(3 * s + 2) = x.b;
}

// Model read of label l at ordinal o with tangents for underlying g.
template <int D>
__device__ __forceinline__ TV model_read(int o, int l, int g, const float2 *R, const ModelDev &m,
                                         const Layout &lay, const float (&S0)[D], float sig_g) {
  l = l < D ? l : 0;
  if (o > 0) {
    const float2 s = SL(lay.off_win + (o & (lay.win - 1)) * D + l);
    if (l != g) return tv(s);
    const float2 x = SL(lay.off_xwin + (o & (lay.win - 1)) * D + l);
    const float st = __fmul_rn(sig_g, __ldg(m.tau + o));
    return {s, scl2(s, __frcp_rn(S0[l])), f2(__fmul_rn(s.x, __fsub_rn(x.x, st)), __fmul_rn(s.y, __fsub_rn(x.y, st)))};
  }
  const float v = __ldg(m.sval + (o + m.n_hist) * D + l);
  TV r = tv(f2(v, v));
  if (o == 0 && l == g) r.a = f2(1.f, 1.f);
  return r;
}

// Dates up to o with the window of X = L W beside S, out of line (for a
// specialised evaluator with many reading instructions).
template <int D>
__device__ __noinline__ void advance_dates_x(int o, PathState<D> &ps, const ModelDev &m, const Layout &lay,
                                             const Rng2 &g, float2 *R, const float (&Bm)[D * D],
                                             const float (&S0)[D], const float (&Lm)[D * D]) {
  while (ps.f < o) gen_date<D, true>(ps.f + 1, ps, m, lay, g, R, Bm, S0, Lm);
}

// X_LRED / X_LANY with tangents (comparisons give zero tangents; min and
// max carry the tangent of the operand they select, the first on ties).
template <int D>
__device__ __forceinline__ TV fused_tv(const uint4 &I, int o, const float *pool, const float2 *R,
                                       const ModelDev &m, const Layout &lay, const float (&S0)[D],
                                       int g, float sig_g) {
  const uint32_t A = I.x >> 8;
  const int n = int((A >> 8) & 3u) + 1, kind = int((A >> 2) & 3u), code = int((A >> 4) & 7u);
  const bool any = (I.x & 0xffu) == X_LANY, conj = (A & 1u) != 0;
  const int rop = int(A & 3u);
  const float k = __uint_as_float(I.w);
  TV v = tv(f2(0.f, 0.f));
  for (int i = 0; i < n; ++i) {
    TV s = model_read<D>(o, int(A >> (10 + 2 * i)) & 3, g, R, m, lay, S0, sig_g);
    if (kind == 1) {
      const float c = pool[I.z + i];
      s = {scl2(s.v, c), scl2(s.a, c), scl2(s.b, c)};
    } else if (kind == 2) {
      const float c = pool[I.z + i];
      s = {f2(__fdiv_rn(s.v.x, c), __fdiv_rn(s.v.y, c)), f2(__fdiv_rn(s.a.x, c), __fdiv_rn(s.a.y, c)),
           f2(__fdiv_rn(s.b.x, c), __fdiv_rn(s.b.y, c))};
    }
    if (any) {
      const float2 p = f2(cmp_code(code, s.v.x, k), cmp_code(code, s.v.y, k));
      if (i == 0) v.v = p;
      else if (conj) v.v = fl2(bits(v.v.x) & bits(p.x), bits(v.v.y) & bits(p.y));
      else v.v = fl2(bits(v.v.x) | bits(p.x), bits(v.v.y) | bits(p.y));
    } else if (i == 0) {
      v = s;
    } else if (rop == 2) {
      v = {add2(v.v, s.v), add2(v.a, s.a), add2(v.b, s.b)};
    } else {
      const bool t0 = rop == 0 ? s.v.x < v.v.x : s.v.x > v.v.x;
      const bool t1 = rop == 0 ? s.v.y < v.v.y : s.v.y > v.v.y;
      if (t0) { v.v.x = s.v.x; v.a.x = s.a.x; v.b.x = s.b.x; }
      if (t1) { v.v.y = s.v.y; v.a.y = s.a.y; v.b.y = s.b.y; }
    }
  }
  if (any) return tv(v.v);
  if (code) return tv(f2(cmp_code(code, v.v.x, k), cmp_code(code, v.v.y, k)));
  return v;
}

// The payoff program with tangents, two paths per lane, warp in step.
template <int D>
__device__ TV eval_greeks(const uint4 *P, const float *pool, float2 *R, const PriceArgs &a,
                          const Rng2 &g, bool live0, bool live1, const float (&Bm)[D * D],
                          const float (&S0)[D], const float (&Lm)[D * D], int gl, float sig_g) {
#include "pc_greeks_state.inc"
  for (;;) {
    const uint4 I = P[pc];
    const uint32_t op = I.x & 0xffu;
    const float kk = __uint_as_float(I.y);
#include "pc_greeks_ops.inc"
  }
}

// The sensitivity launch for underlying g = a.greek_label, generic in the
// tangent evaluator EVAL(P, pool, R, g, live0, live1, Bm, S0, Lm, g, sig_g)
// (the interpreter eval_greeks, or a run-time specialised evaluator): per
// path (x, dx/dS0_g, dx/dsigma_g); per tile the FP64 sums and sums of
// squares of the three, in the pricing kernel's deterministic chunked
// reduction (width 6).
template <int D, bool WRITE, typename EVAL>
__device__ __forceinline__ void greeks_tiles(const PriceArgs &a, EVAL eval) {
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
  const int gl = a.greek_label;
  const float sig_g = __ldg(a.m.sig + gl);
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
    const TV x = eval(P, pool, R, g, live0, live1, Bm, S0, Lm, gl, sig_g);
    Moments<6> mo;
    const float q0[3] = {x.v.x, x.a.x, x.b.x}, q1[3] = {x.v.y, x.a.y, x.b.y};
    if (live0) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        mo.add(2 * j, q0[j]);
        mo.add_prod(2 * j + 1, q0[j], q0[j]);
        if (WRITE) a.out_paths[i0 * 3 + j] = q0[j];
      }
    }
    if (live1) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        mo.add(2 * j, q1[j]);
        mo.add_prod(2 * j + 1, q1[j], q1[j]);
        if (WRITE) a.out_paths[i1 * 3 + j] = q1[j];
      }
    }
    double tp[6];
    mo.warp_total(tp);
    finish_tile<6>(a, tile, tp, lane);
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
