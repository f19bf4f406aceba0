// pc_cv.cuh -- the control-variate pricing kernel's body (cv_tiles), generic
// in the payoff evaluator (the interpreter eval_path, or a run-time
// specialised evaluator), with the hedge-ratio table interpolation and the
// hedge gains.  Included by pc_cv.cu and by the run-time compiler.
//
// For the worst-of autocallable template each path's payoff X comes from the
// evaluator exactly as in the pricing kernel; as the evaluator generates each
// date, the kernel accumulates the discounted hedge gains
//   M = sum_{k<n} alive_k sum_i Delta_i(k) (D_{k+1} S_i(t_{k+1}) - D_k S_i(t_k))
// with Delta from a table over ln S (multilinear interpolation) per date and
// knock-in state.  Every factor of a term is known at t_k, so E[M] = 0.  An
// optional second-order term M2 (gamma from the table's slopes, the
// quadratic moments of the discounted returns in closed form) also has mean
// zero, and Y = X - beta M - beta2 M2 estimates the same price for any fixed
// betas.  The tile sums carry X, X^2, Y, Y^2, or in the pilot mode the
// eight first and second moments of X, M, M2 that the variance-minimising
// betas need.
// A hedge period whose end date the warp never generated (every lane's
// program stopped before it) is skipped: that decision depends only on
// information at t_k of this and of independent paths, so the terms kept are
// still martingale increments.
#pragma once

#include "pc_device.cuh"
#include "pc_cv_types.h"

namespace pc {

// Hedge ratios at ln S (given as l2 = log2 S: the axis coordinate is
// u = l2 ln2 / h - lo / h, clamped to the grid) from the nearest table node
// a = floor(u + 1/2): its ratios plus the first-order step along its slopes,
// Delta_i = Delta_i(a) + sum_j s_ij(a) (u_j - a_j); with SLOPES also the
// slopes s[i][j] = d Delta_i / d u_j (the node's).  A node is kCvRecord
// floats (ratios, then s_ij at 3 + 3 i + j): one to three 16-byte loads.
template <int D, bool SLOPES>
__device__ __forceinline__ void table_delta(const CvArgs &c, int k, int ki, const float (&l2)[D],
                                            float (&delta)[D], float (&s)[D][D]) {
  const float4 *tab = reinterpret_cast<const float4 *>(c.tables) +
                      (size_t(k - 1) * 2 + ki) * size_t(c.nodes) * (kCvRecord / 4);
  const int G = c.grid;
  int node = 0;
  float f[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float u = fmaf(l2[i], c.ua[k - 1][i], -c.ub[k - 1][i]);
    u = fminf(fmaxf(u, 0.f), float(G - 1));
    const float a = floorf(u + 0.5f);
    f[i] = u - a;
    node = node * G + int(a);
  }
  constexpr int NV = D == 1 ? 1 : D == 2 ? 2 : 3;  // float4s holding slots 0 .. 3 + 3 (D - 1) + D - 1
  float r[4 * NV];
  const float4 *rec = tab + size_t(node) * (kCvRecord / 4);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float4 x = __ldg(rec + v);
    r[4 * v] = x.x;
    r[4 * v + 1] = x.y;
    r[4 * v + 2] = x.z;
    r[4 * v + 3] = x.w;
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float di = r[i];
#pragma unroll
    for (int jj = 0; jj < D; ++jj) {
      const float sij = r[3 + 3 * i + jj];
      di = fmaf(sij, f[jj], di);
      if (SLOPES) s[i][jj] = sij;
    }
    delta[i] = di;
  }
}

// Hedge gains of the lane's two paths (q = 0, 1), accumulated online: the
// evaluators call on_date(t, read) after generating date t, and the period
// k = t - 1 (from t_k to t_{k+1}) is added then, from S at t_k (kept here)
// and S at t_{k+1} (read from the evaluator).  A period whose end date the
// warp never generates is never added.  First order M and second order M2;
// a dead path's terms are computed and discarded, a period in which both
// are dead is skipped.
template <int D, bool GAMMA>
struct CvOnline {
  static constexpr bool kNone = false;
  const CvArgs &c;
  const ModelDev &m;
  float sk[2][D];  // S at t_k (t_0: the spot)
  float M[2], M2[2];
  bool alive[2];
  int ki[2];

  __device__ __forceinline__ CvOnline(const CvArgs &c_, const ModelDev &m_, const float (&S0)[D])
      : c(c_), m(m_) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
      for (int i = 0; i < D; ++i) sk[q][i] = S0[i];
      M[q] = M2[q] = 0.f;
      alive[q] = true;
      ki[q] = 0;
    }
  }

  template <class RD>
  __device__ __forceinline__ void on_date(int t, RD &read) {
    const int k = t - 1;
    if (k >= c.n) return;
    float sn[2][D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float2 v = read(t, i);
      sn[0][i] = v.x;
      sn[1][i] = v.y;
    }
    period(k, sn);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int i = 0; i < D; ++i) sk[q][i] = sn[q][i];
  }

  __device__ __forceinline__ void period(int k, const float (&sn)[2][D]) {
    if (k >= 1) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float worst = sk[q][0] * c.inv_ref[0];
#pragma unroll
        for (int i = 1; i < D; ++i) worst = fminf(worst, sk[q][i] * c.inv_ref[i]);
        ki[q] |= worst <= c.ki_level ? 1 : 0;
        alive[q] = alive[q] && !(worst >= c.call_level);
      }
    }
    if (!alive[0] && !alive[1]) return;
    const float d0 = __ldg(m.disc + k + m.n_hist), d1 = __ldg(m.disc + k + 1 + m.n_hist);
    // one path at a time (a rolled loop over register selects): the
    // evaluator's state is live around this call, so only one path's corner
    // values are held at once
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
      float s0[D], s1[D], delta[D], sl[D][D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        s0[i] = q ? sk[1][i] : sk[0][i];
        s1[i] = q ? sn[1][i] : sn[0][i];
      }
      const bool al = q ? alive[1] : alive[0];
      if (k == 0) {
#pragma unroll
        for (int i = 0; i < D; ++i) delta[i] = c.delta0_dev ? __ldg(c.delta0_dev + i) : c.delta0[i];
      } else {
        float l2[D];
#pragma unroll
        for (int i = 0; i < D; ++i) l2[i] = __log2f(s0[i]);
        table_delta<D, GAMMA>(c, k, q ? ki[1] : ki[0], l2, delta, sl);
      }
      float X[D];
      float dm = 0.f;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        X[i] = d1 * s1[i] - d0 * s0[i];
        dm = fmaf(delta[i], X[i], dm);
      }
      const float dM = al ? dm : 0.f;
      if (q) M[1] += dM;
      else M[0] += dM;
      if (GAMMA && k >= 1) {
        // Gamma = sym(t), t_ij = s_ij / (h_j S_j); the quadratic forms of
        // a symmetric weight need only t itself.  1 / (h_j S_j) with the
        // approximate reciprocal: any hedge ratio known at t_k keeps the
        // term's mean zero, so the weights need no exact rounding.
        float wj[D];
#pragma unroll
        for (int j = 0; j < D; ++j) wj[j] = __fdividef(c.inv_h[k - 1][j], s0[j]);
        float qf = 0.f, e = 0.f;
#pragma unroll
        for (int i = 0; i < D; ++i) {
          float rq = 0.f, re = 0.f;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            const float tt = sl[i][j] * wj[j];
            rq = fmaf(tt, X[j], rq);
            re = fmaf(tt, s0[j] * c.cq[k][i * kCvMaxD + j], re);
          }
          qf = fmaf(X[i], rq, qf);
          e = fmaf(s0[i], re, e);
        }
        const float dM2 = al ? 0.5f * (qf - d0 * d0 * e) : 0.f;
        if (q) M2[1] += dM2;
        else M2[0] += dM2;
      }
    }
  }
};

// EVAL(P, pool, R, g, live0, live1, Bm, S0, &hook) -> float2 payoffs of the
// lane's two paths; the evaluator calls hook.on_date after each date.
template <int D, int MODE, typename EVAL>
__device__ __forceinline__ void cv_tiles(const PriceArgs &a, const CvArgs &c, EVAL eval) {
  constexpr bool WRITE = (MODE & kCvWrite) != 0, GAMMA = (MODE & kCvGamma) != 0,
                 PILOT = (MODE & kCvPilot) != 0;
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
    CvOnline<D, GAMMA> hg(c, a.m, S0);
    const float2 x = eval(P, pool, R, g, live0, live1, Bm, S0, &hg);
    const float(&Mv)[2] = hg.M;
    const float(&M2v)[2] = hg.M2;
    const float xs[2] = {x.x, x.y};
    const bool live[2] = {live0, live1};
    if (WRITE) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!live[q]) continue;
        const uint64_t i = q ? i1 : i0;
        a.out_paths[3 * i] = xs[q];
        a.out_paths[3 * i + 1] = Mv[q];
        a.out_paths[3 * i + 2] = M2v[q];
      }
    }
    if (PILOT) {
      Moments<8> mo;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!live[q]) continue;
        mo.add(0, xs[q]);
        mo.add(1, Mv[q]);
        mo.add(2, M2v[q]);
        mo.add_prod(3, xs[q], Mv[q]);
        mo.add_prod(4, xs[q], M2v[q]);
        mo.add_prod(5, Mv[q], Mv[q]);
        mo.add_prod(6, M2v[q], M2v[q]);
        mo.add_prod(7, Mv[q], M2v[q]);
      }
      double tp[8];
      mo.warp_total(tp);
      finish_tile<8>(a, tile, tp, lane);
    } else {
      Moments<4> mo;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!live[q]) continue;
        const float y = xs[q] - c.beta * Mv[q] - c.beta2 * M2v[q];
        mo.add(0, xs[q]);
        mo.add_prod(1, xs[q], xs[q]);
        mo.add(2, y);
        mo.add_prod(3, y, y);
      }
      double tp[4];
      mo.warp_total(tp);
      finish_tile<4>(a, tile, tp, lane);
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

}  // namespace pc
