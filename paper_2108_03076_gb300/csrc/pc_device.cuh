// pc_device.cuh -- device building blocks shared by the pricing kernel
// (pc_kernels.cu) and the pathwise-sensitivity kernel (pc_greeks.cu):
// Philox4x32-10 (Salmon et al., SC'11), 24-bit uniforms, Box-Muller, the
// date-ordered Brownian bridge (normals in the order the walk uses them),
// correlated GBM, the fused multi-asset reads, and the deterministic
// reduction (float-pair tile sums, FP64 chunk sums).
//
// Per-thread state lives in shared memory as word-interleaved slots: slot s
// of thread t is at region[s * blockDim.x + t] (float2: two paths per lane),
// so the warp-uniform slot indices give conflict-free accesses.
#pragma once

#include "pc_types.h"

namespace pc {
namespace {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;
constexpr unsigned kFull = 0xffffffffu;

// 2*pi*u - pi for u = (k + 1/2) 2^-24, as one FMA in k.
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float kThetaScale = float(kTwoPi / 16777216.0);
constexpr float kThetaOffset = float(kTwoPi / 33554432.0 - kTwoPi / 2.0);

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed FP32 pairs (f32x2): one instruction for both paths of a lane; each
// half is rounded as the scalar operation rounds it, so results are those
// of two scalar operations.
__device__ __forceinline__ float2 fma_x2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 mul_x2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// Philox4x32-10: ten rounds of two 32x32->64 multiplies, the key bumped by
// the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// The same with the round keys precomputed (rk[2r], rk[2r + 1]: PriceArgs):
// no key arithmetic, and in a kernel parameter the keys come from the
// constant bank.
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint32_t *rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Box-Muller on one word pair of each of the lane's two paths: u_a from the
// even word, u_b from the odd word (path 0 in .x, path 1 in .y); even normal
// r cos(2 pi u_b), odd normal r sin(2 pi u_b) with r = sqrt(q), q = -2 ln u_a.
// u = (k + 1/2) 2^-24 for the 24-bit integer k = word >> 8.  Away from u = 1,
// q = -2 ln 2 lg2.approx(u), whose absolute error (about 7e-8 over (0, 1)) is
// small beside q.  Near 1, where q is tiny and both that error and the
// rounding of u to a float would dominate, q is the series 2v + v^2 +
// (2/3) v^3 of -2 ln(1 - v) in v = 1 - u, which is exact in float for
// u > 1/2 (an odd multiple of 2^-25 below 2^-1); for v < 2^-8 the terms left
// out are below 2^-26 of q.  The angle is reduced to 2 pi u_b - pi in
// (-pi, pi), where cos and sin change sign.  The scalar steps run on packed
// pairs (each lane of a packed operation rounds as the scalar one).
__device__ __forceinline__ void box_muller2(uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1,
                                            float2 &ze, float2 &zo) {
  const float2 ka = make_float2(__uint2float_rn(a0 >> 8), __uint2float_rn(a1 >> 8));
  const float2 u = fma_x2(ka, dup2(0x1p-24f), dup2(0x1p-25f));
  const float2 v = fma_x2(fma_x2(ka, dup2(-0x1p-24f), dup2(1.0f)), dup2(1.0f), dup2(-0x1p-25f));
  const float2 ql = mul_x2(dup2(-1.3862943611198906f), make_float2(lg2_approx(u.x), lg2_approx(u.y)));
  const float2 qs = mul_x2(v, fma_x2(v, fma_x2(v, dup2(0.6666666666666666f), dup2(1.0f)), dup2(2.0f)));
  const float2 q = make_float2(v.x < 0x1p-8f ? qs.x : ql.x, v.y < 0x1p-8f ? qs.y : ql.y);
  const float2 nr = make_float2(-sqrt_approx(q.x), -sqrt_approx(q.y));
  const float2 kb = make_float2(__uint2float_rn(b0 >> 8), __uint2float_rn(b1 >> 8));
  const float2 th = fma_x2(kb, dup2(kThetaScale), dup2(kThetaOffset));
  ze = mul_x2(nr, make_float2(cos_approx(th.x), cos_approx(th.y)));
  zo = mul_x2(nr, make_float2(sin_approx(th.x), sin_approx(th.y)));
}

// Two paths per lane: every value of the stack machine is a float2 (.x for
// the lane's first path, .y for its second), so each fetched and decoded
// instruction does the work of two paths and the two independent dependency
// chains (Philox rounds, Box-Muller, bridge) overlap in the pipeline.
// A lane with H pairs of paths (H = 2 in a specialised kernel with four
// paths per lane) keeps the counters of its 2H paths.
template <int H>
struct RngH {
  uint32_t plo[2 * H], phi[2 * H];
  uint32_t stream;
  uint32_t rk[20];  // Philox round keys (PriceArgs::rk), copied: the compiler keeps them uniform
};
using Rng2 = RngH<1>;

// The four normals of Philox block b of both paths.
__device__ __forceinline__ void block_normals2(uint32_t b, const Rng2 &g, float2 (&e)[4]) {
  const uint4 x0 = philox_rk(make_uint4(b, g.plo[0], g.phi[0], g.stream), g.rk);
  const uint4 x1 = philox_rk(make_uint4(b, g.plo[1], g.phi[1], g.stream), g.rk);
  box_muller2(x0.x, x0.y, x1.x, x1.y, e[0], e[1]);
  box_muller2(x0.z, x0.w, x1.z, x1.w, e[2], e[3]);
}

// The same for each pair h of a lane's 2H paths.
template <int H>
__device__ __forceinline__ void block_normals_h(uint32_t b, const RngH<H> &g, float2 (&e)[H][4]) {
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const uint4 x0 = philox_rk(make_uint4(b, g.plo[2 * h], g.phi[2 * h], g.stream), g.rk);
    const uint4 x1 = philox_rk(make_uint4(b, g.plo[2 * h + 1], g.phi[2 * h + 1], g.stream), g.rk);
    box_muller2(x0.x, x0.y, x1.x, x1.y, e[h][0], e[h][1]);
    box_muller2(x0.z, x0.w, x1.z, x1.w, e[h][2], e[h][3]);
  }
}

// Slot s of this thread in the word-interleaved per-thread region (the
// stride is the block size, 32..kBlock threads; a run-time specialised
// kernel is compiled for its block size, so its slot offsets are constants).
#ifdef PC_SLOT_STRIDE
#define SL(s) R[(s) * PC_SLOT_STRIDE]
#else
#define SL(s) R[(s) * blockDim.x]
#endif

// Window slot w (0 .. win * d - 1) of this thread: in the shared region
// (word-interleaved after lay.off_win) or, with GW, in the thread's column
// of the HBM window (coalesced across the warp for a uniform slot).
template <bool GW>
__device__ __forceinline__ float2 win_load(const float2 *R, const Layout &lay, int w) {
  if constexpr (GW)
    return lay.gwin[int64_t(w) * lay.gstride + int64_t(blockIdx.x) * blockDim.x + threadIdx.x];
  else
    return SL(lay.off_win + w);
}
template <bool GW>
__device__ __forceinline__ void win_store(float2 *R, const Layout &lay, int w, float2 v) {
  if constexpr (GW)
    lay.gwin[int64_t(w) * lay.gstride + int64_t(blockIdx.x) * blockDim.x + threadIdx.x] = v;
  else
    SL(lay.off_win + w) = v;
}

// Per-path state of a lane's H pairs of paths; the bridge stack holds, per
// level, the D values of pair 0, then of pair 1 (D H slots a level).
template <int D, int H = 1>
struct PathState {
  float2 w[H][D];               // W at the last produced date
  float2 zc[H][3];              // words 1..3 of the last Philox block (d < 4)
  int f;                        // last produced ordinal (frontier), warp-uniform
  int bsp;                      // bridge stack size, warp-uniform
  int k;                        // ops run so far (the next op's number), warp-uniform
#ifdef PC_WIN_REGS
  float2 s[H][D];               // S at the frontier date: the whole window of a program
                                // that reads no date behind the frontier
#endif
};

// A path's state at its start; the bottom level of the bridge stack is
// zeroed (the root op reads it with weight 0).
template <int D, int H>
__device__ __forceinline__ void path_state_init(PathState<D, H> &ps, float2 *R, const Layout &lay) {
#pragma unroll
  for (int i = 0; i < D * H; ++i) SL(lay.off_bstack + i) = make_float2(0.f, 0.f);
#pragma unroll
  for (int h = 0; h < H; ++h) {
#pragma unroll
    for (int i = 0; i < D; ++i) ps.w[h][i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 3; ++i) ps.zc[h][i] = make_float2(0.f, 0.f);
  }
  ps.f = 0;
  ps.bsp = 0;
  ps.k = 0;
}

// The normals of op k for every path of the lane: normals D k .. D k + D - 1
// of the path (Philox block m >> 2, word m & 3).  Ops run in order, so the
// block holding normal D k is either new or the last block computed, whose
// words 1..3 the state keeps (zc); a new block is computed at most once per
// op.
template <int D, int H>
__device__ __forceinline__ void node_normals(uint32_t k, const RngH<H> &g, float2 (&zc)[H][3],
                                             float2 (&z)[H][D]) {
  if constexpr (D == 4) {
    float2 e[H][4];
    block_normals_h<H>(k, g, e);
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
      for (int i = 0; i < 4; ++i) z[h][i] = e[h][i];
  } else if constexpr (D == 2) {
    if (k & 1) {  // words 2, 3 of block k / 2
#pragma unroll
      for (int h = 0; h < H; ++h) {
        z[h][0] = zc[h][1];
        z[h][1] = zc[h][2];
      }
    } else {
      float2 e[H][4];
      block_normals_h<H>(k >> 1, g, e);
#pragma unroll
      for (int h = 0; h < H; ++h) {
        z[h][0] = e[h][0];
        z[h][1] = e[h][1];
        zc[h][1] = e[h][2];
        zc[h][2] = e[h][3];
      }
    }
  } else if constexpr (D == 1) {
    const uint32_t ph = k & 3;
    if (ph == 0) {
      float2 e[H][4];
      block_normals_h<H>(k >> 2, g, e);
#pragma unroll
      for (int h = 0; h < H; ++h) {
        z[h][0] = e[h][0];
        zc[h][0] = e[h][1];
        zc[h][1] = e[h][2];
        zc[h][2] = e[h][3];
      }
    } else {
#pragma unroll
      for (int h = 0; h < H; ++h) z[h][0] = ph == 1 ? zc[h][0] : ph == 2 ? zc[h][1] : zc[h][2];
    }
  } else {  // D == 3: the first normal is word ph = 3k & 3 of its block
    const uint32_t ph = (3 * k) & 3;
    if (ph == 1) {  // words 1..3 of the last block
#pragma unroll
      for (int h = 0; h < H; ++h) {
        z[h][0] = zc[h][0];
        z[h][1] = zc[h][1];
        z[h][2] = zc[h][2];
      }
    } else {
      float2 e[H][4];
      block_normals_h<H>((3 * k + 2) >> 2, g, e);
#pragma unroll
      for (int h = 0; h < H; ++h) {
        if (ph == 0) {
          z[h][0] = e[h][0];
          z[h][1] = e[h][1];
          z[h][2] = e[h][2];
        } else if (ph == 2) {
          z[h][0] = zc[h][1];
          z[h][1] = zc[h][2];
          z[h][2] = e[h][0];
        } else {
          z[h][0] = zc[h][2];
          z[h][1] = e[h][0];
          z[h][2] = e[h][1];
        }
        zc[h][0] = e[h][1];
        zc[h][1] = e[h][2];
        zc[h][2] = e[h][3];
      }
    }
  }
}

// A bridge op's weights as packed pairs (two 16-byte loads through the
// read-only path: the address is the same in every lane).
struct OpRegs {
  float2 wl, wr, sd;
};
__device__ __forceinline__ OpRegs load_op(const BridgeOp *p) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
  const float4 a = __ldg(q), b = __ldg(q + 1);
  OpRegs o;
  o.wl = make_float2(a.x, a.y);
  o.wr = make_float2(a.z, a.w);
  o.sd = make_float2(b.x, b.y);
  return o;
}

// Produce date t (= frontier + 1) for the lane's paths: bridge ops of t,
// then GBM into the window slot of t.  With XW the correlated Brownian
// values X = L W of the date are also kept (window at lay.off_xwin), which
// the pathwise sensitivities need.  The bridge, correlation and GBM products
// run on packed pairs (two paths of the lane); with H pairs a lane, each op's
// schedule and control serve all 2H paths.
template <int D, bool XW = false, bool GW = false, int H = 1>
__device__ __forceinline__ void gen_date(int t, PathState<D, H> &ps, const ModelDev &m,
                                         const Layout &lay, const RngH<H> &g, float2 *R,
                                         const float (&Bm)[D * D], const float (&S0)[D],
                                         const float *Lm = nullptr) {
  static_assert(H == 1 || (!XW && !GW), "several path pairs a lane: no X window, no HBM window");
  const int k1 = __ldg(m.date_ops + t + 1);  // ops of date t: [ps.k, k1)
  // Every op pushes its node; the date's own value (the last node, or one
  // pushed on an earlier date when t has no op) is then popped as the new
  // frontier value.  The root op has wl = wr = 0 and reads the bottom level,
  // zeroed at the path's start, as its right end.  (Branch-free: a push or
  // keep decision per op, and a root test, cost register moves at the joins.)
  for (; ps.k < k1; ++ps.k) {
    const OpRegs op = load_op(m.ops + ps.k);
    float2 z[H][D];
    node_normals<D, H>(uint32_t(ps.k), g, ps.zc, z);
    const int top = lay.off_bstack + max(ps.bsp - 1, 0) * D * H;
    const int nxt = lay.off_bstack + ps.bsp * D * H;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      float2 nw[D];
#pragma unroll
      for (int i = 0; i < D; ++i)
        nw[i] = fma_x2(op.wl, ps.w[h][i], fma_x2(op.wr, SL(top + h * D + i), mul_x2(op.sd, z[h][i])));
#pragma unroll
      for (int i = 0; i < D; ++i) SL(nxt + h * D + i) = nw[i];
    }
    ++ps.bsp;
  }
  --ps.bsp;
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int i = 0; i < D; ++i) ps.w[h][i] = SL(lay.off_bstack + ps.bsp * D * H + h * D + i);
  const int ws = (t & (lay.win - 1)) * D;
#pragma unroll
  for (int h = 0; h < H; ++h) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float2 x = __ldg(m.A + t * D + i);
#pragma unroll
      for (int k = 0; k <= i; ++k)
        x = make_float2(fmaf(Bm[i * D + k], ps.w[h][k].x, x.x), fmaf(Bm[i * D + k], ps.w[h][k].y, x.y));
#ifdef PC_WIN_REGS
      ps.s[h][i] = make_float2(S0[i] * ex2_approx(x.x), S0[i] * ex2_approx(x.y));
      (void)ws;
#else
      win_store<GW>(R, lay, ws + i, make_float2(S0[i] * ex2_approx(x.x), S0[i] * ex2_approx(x.y)));
#endif
    }
  }
  if constexpr (XW) {
    const int xs = lay.off_xwin + (t & (lay.win - 1)) * D;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float2 x = mul_x2(dup2(Lm[i * D]), ps.w[0][0]);
#pragma unroll
      for (int k = 1; k <= i; ++k) x = fma_x2(dup2(Lm[i * D + k]), ps.w[0][k], x);
      SL(xs + i) = x;
    }
  }
  ps.f = t;
}

// The evaluators' per-date hook: called after each generated date t with
// the evaluator's reader (read(t, i): S_i at ordinal t of the lane's paths).
// NoDateHook (pricing) does nothing; the control-variate kernel's hook
// accumulates its hedge gains there.
struct NoDateHook {
  static constexpr bool kNone = true;
  template <class RD>
  __device__ __forceinline__ void on_date(int, RD &) {}
};

// Dates ps.f + 1 .. o, out of line (the specialised evaluator calls it from
// every instruction that reads a date, so it is not inlined there).
template <int D, bool GW, int H>
__device__ __noinline__ void advance_dates(int o, PathState<D, H> &ps, const ModelDev &m, const Layout &lay,
                                           const RngH<H> &g, float2 *R, const float (&Bm)[D * D],
                                           const float (&S0)[D]) {
  while (ps.f < o) gen_date<D, false, GW>(ps.f + 1, ps, m, lay, g, R, Bm, S0);
}

template <int D>
__device__ __forceinline__ void load_model_regs(const ModelDev &m, float (&Bm)[D * D],
                                                float (&S0)[D]) {
#pragma unroll
  for (int i = 0; i < D * D; ++i) Bm[i] = m.Bv[i];
#pragma unroll
  for (int i = 0; i < D; ++i) S0[i] = m.S0v[i];
}

__device__ __forceinline__ int bits(float v) { return __float_as_int(v); }
__device__ __forceinline__ float fl(int v) { return __int_as_float(v); }
__device__ __forceinline__ float2 fl2(int a, int b) { return make_float2(fl(a), fl(b)); }

__device__ __forceinline__ float cmp_code(int code, float v, float k) {
  // 1: v < k, 2: v <= k, 3: k < v, 4: k <= v
  const bool r = code == 1 ? v < k : code == 2 ? v <= k : code == 3 ? k < v : k <= v;
  return fl(int(r));
}

// Fused multi-asset value (X_LRED) or test (X_LANY) of instruction I at
// ordinal o for both paths; results of compares are 0/1 int bits.
// rd(l): S of underlying l at o (o > 0).
template <int D, typename RD>
__device__ __forceinline__ float2 fused_value_rd(const uint4 &I, int o, const float *pool, const ModelDev &m,
                                                 RD rd) {
  const uint32_t A = I.x >> 8;
  const int n = int((A >> 8) & 3u) + 1, kind = int((A >> 2) & 3u), code = int((A >> 4) & 7u);
  const bool any = (I.x & 0xffu) == X_LANY, conj = (A & 1u) != 0;
  const int rop = int(A & 3u);
  const float k = __uint_as_float(I.w);
  float2 v = make_float2(0.f, 0.f);
  for (int i = 0; i < n; ++i) {
    int l = int(A >> (10 + 2 * i)) & 3;
    l = l < D ? l : 0;
    float2 s;
    if (o > 0) {
      s = rd(l);
    } else {
      const float sv = __ldg(m.sval + (o + m.n_hist) * D + l);
      s = make_float2(sv, sv);
    }
    if (kind == 1) {
      const float c = pool[I.z + i];
      s = make_float2(__fmul_rn(s.x, c), __fmul_rn(s.y, c));
    } else if (kind == 2) {
      const float c = pool[I.z + i];
      s = make_float2(__fdiv_rn(s.x, c), __fdiv_rn(s.y, c));
    }
    if (any) {
      const float2 p = make_float2(cmp_code(code, s.x, k), cmp_code(code, s.y, k));
      if (i == 0) v = p;
      else if (conj) v = fl2(bits(v.x) & bits(p.x), bits(v.y) & bits(p.y));
      else v = fl2(bits(v.x) | bits(p.x), bits(v.y) | bits(p.y));
    } else if (i == 0) {
      v = s;
    } else if (rop == 0) {
      v = make_float2(fminf(v.x, s.x), fminf(v.y, s.y));
    } else if (rop == 1) {
      v = make_float2(fmaxf(v.x, s.x), fmaxf(v.y, s.y));
    } else {
      v = make_float2(__fadd_rn(v.x, s.x), __fadd_rn(v.y, s.y));
    }
  }
  if (!any && code) v = make_float2(cmp_code(code, v.x, k), cmp_code(code, v.y, k));
  return v;
}

template <int D, bool GW = false>
__device__ __forceinline__ float2 fused_value(const uint4 &I, int o, const float *pool, const float2 *R,
                                              const ModelDev &m, const Layout &lay) {
  const int base = (o & (lay.win - 1)) * D;
  return fused_value_rd<D>(I, o, pool, m, [&](int l) { return win_load<GW>(R, lay, base + l); });
}
// The same with the frontier date's S in registers (cur; a window of one date).
template <int D>
__device__ __forceinline__ float2 fused_value_regs(const uint4 &I, int o, const float *pool,
                                                   const float2 (&cur)[D], const ModelDev &m) {
  return fused_value_rd<D>(I, o, pool, m, [&](int l) { return cur[l]; });
}

// The same instruction as a test only (X_LANY, or X_LRED with a compare),
// as booleans for the lane's two paths: the whole-loop barrier op decides
// its latches from it without the 0/1 value bits.
template <int D, typename RD>
__device__ __forceinline__ void fused_test_rd(const uint4 &I, int o, const float *pool, const ModelDev &m,
                                              RD rd, bool &t0, bool &t1) {
  const uint32_t A = I.x >> 8;
  const int n = int((A >> 8) & 3u) + 1, kind = int((A >> 2) & 3u), code = int((A >> 4) & 7u);
  const bool any = (I.x & 0xffu) == X_LANY, conj = (A & 1u) != 0;
  const int rop = int(A & 3u);
  const float k = __uint_as_float(I.w);
  auto cmp = [&](float v) {
    return code == 1 ? v < k : code == 2 ? v <= k : code == 3 ? k < v : k <= v;
  };
  float2 v = make_float2(0.f, 0.f);
  bool b0 = false, b1 = false;
  for (int i = 0; i < n; ++i) {
    int l = int(A >> (10 + 2 * i)) & 3;
    l = l < D ? l : 0;
    float2 s;
    if (o > 0) {
      s = rd(l);
    } else {
      const float sv = __ldg(m.sval + (o + m.n_hist) * D + l);
      s = make_float2(sv, sv);
    }
    if (kind == 1) {
      const float c = pool[I.z + i];
      s = make_float2(__fmul_rn(s.x, c), __fmul_rn(s.y, c));
    } else if (kind == 2) {
      const float c = pool[I.z + i];
      s = make_float2(__fdiv_rn(s.x, c), __fdiv_rn(s.y, c));
    }
    if (any) {
      const bool p0 = cmp(s.x), p1 = cmp(s.y);
      if (i == 0) {
        b0 = p0;
        b1 = p1;
      } else if (conj) {
        b0 = b0 && p0;
        b1 = b1 && p1;
      } else {
        b0 = b0 || p0;
        b1 = b1 || p1;
      }
    } else if (i == 0) {
      v = s;
    } else if (rop == 0) {
      v = make_float2(fminf(v.x, s.x), fminf(v.y, s.y));
    } else if (rop == 1) {
      v = make_float2(fmaxf(v.x, s.x), fmaxf(v.y, s.y));
    } else {
      v = make_float2(__fadd_rn(v.x, s.x), __fadd_rn(v.y, s.y));
    }
  }
  if (!any) {
    b0 = cmp(v.x);
    b1 = cmp(v.y);
  }
  t0 = b0;
  t1 = b1;
}
template <int D, bool GW = false>
__device__ __forceinline__ void fused_test(const uint4 &I, int o, const float *pool, const float2 *R,
                                           const ModelDev &m, const Layout &lay, bool &t0, bool &t1) {
  const int base = (o & (lay.win - 1)) * D;
  fused_test_rd<D>(I, o, pool, m, [&](int l) { return win_load<GW>(R, lay, base + l); }, t0, t1);
}
template <int D>
__device__ __forceinline__ void fused_test_regs(const uint4 &I, int o, const float *pool, const float2 (&cur)[D],
                                                const ModelDev &m, bool &t0, bool &t1) {
  fused_test_rd<D>(I, o, pool, m, [&](int l) { return cur[l]; }, t0, t1);
}

// Values of the stack machine: one per path of the lane, kPL = 2 PC_PAIRS of
// them (PC_PAIRS pairs; a specialised kernel with four paths a lane defines
// PC_PAIRS 2).  pv_get / pv_set take a path index that is a constant once the
// loops over it are unrolled.
#ifndef PC_PAIRS
#define PC_PAIRS 1
#endif
constexpr int kPL = 2 * PC_PAIRS;
#if PC_PAIRS == 2
struct PV {
  float2 a, b;
};
__device__ __forceinline__ float pv_get(const PV &v, int p) {
  return p == 0 ? v.a.x : p == 1 ? v.a.y : p == 2 ? v.b.x : v.b.y;
}
__device__ __forceinline__ void pv_set(PV &v, int p, float x) {
  if (p == 0) v.a.x = x;
  else if (p == 1) v.a.y = x;
  else if (p == 2) v.b.x = x;
  else v.b.y = x;
}
__device__ __forceinline__ PV pv_splat(float x) { return PV{make_float2(x, x), make_float2(x, x)}; }
__device__ __forceinline__ PV pv_pairs(float2 p0, float2 p1) { return PV{p0, p1}; }
#else
typedef float2 PV;
__device__ __forceinline__ float pv_get(const PV &v, int p) { return p ? v.y : v.x; }
__device__ __forceinline__ void pv_set(PV &v, int p, float x) {
  if (p) v.y = x;
  else v.x = x;
}
__device__ __forceinline__ PV pv_splat(float x) { return make_float2(x, x); }
__device__ __forceinline__ PV pv_pairs(float2 p0) { return p0; }
#endif
#define PV_FOR(p) _Pragma("unroll") for (int p = 0; p < kPL; ++p)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// A tile's moment sums (sum of payoffs, of squares, of products) without
// the FP64 pipe, which issues at a small fraction of the FP32 rate here:
// each sum is an unevaluated pair hi + lo of floats.  An addend enters by
// Knuth's two-sum (hi + x = s + e exactly, e added into lo); a product of
// two floats enters exactly as its rounded value plus the FMA residual.
// Only the low parts round, so a warp's 64-path sums carry a relative
// error of order 2^-45 of the sum of magnitudes (an FP64 sum of the same
// terms: 2^-47), and become doubles once per tile for the chunk sums.
template <int W>
struct Moments {
  float hi[W], lo[W];
  __device__ __forceinline__ Moments() {
#pragma unroll
    for (int v = 0; v < W; ++v) hi[v] = lo[v] = 0.f;
  }
  __device__ __forceinline__ void add(int v, float x) {
    const float s = __fadd_rn(hi[v], x);
    const float b = __fsub_rn(s, hi[v]);
    const float e = __fadd_rn(__fsub_rn(hi[v], __fsub_rn(s, b)), __fsub_rn(x, b));
    hi[v] = s;
    lo[v] = __fadd_rn(lo[v], e);
  }
  __device__ __forceinline__ void add_prod(int v, float x, float y) {
    const float p = __fmul_rn(x, y);
    add(v, p);
    lo[v] = __fadd_rn(lo[v], __fmaf_rn(x, y, -p));
  }
  // warp totals (identical in every lane: the butterfly's additions are
  // commutative) as doubles
  __device__ __forceinline__ void warp_total(double (&tp)[W]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int v = 0; v < W; ++v) {
        const float h = __shfl_xor_sync(kFull, hi[v], o), l = __shfl_xor_sync(kFull, lo[v], o);
        const float s = __fadd_rn(hi[v], h);
        const float b = __fsub_rn(s, hi[v]);
        const float e = __fadd_rn(__fsub_rn(hi[v], __fsub_rn(s, b)), __fsub_rn(h, b));
        hi[v] = s;
        lo[v] = __fadd_rn(__fadd_rn(lo[v], l), e);
      }
    }
#pragma unroll
    for (int v = 0; v < W; ++v) tp[v] = double(hi[v]) + double(lo[v]);
  }
};

// Deterministic reduction.  Tile t's partials (sum, sum of squares, ...) are
// the warp's Moments totals, in a fixed shuffle order, as doubles.  Tiles form chunks of chunk_tiles
// consecutive tiles; the warp that finishes a chunk's last tile sums the
// chunk's partials in index order (lane l takes tiles l, l+32, ...; then a
// fixed shuffle tree), and the warp that finishes the last chunk sums the
// chunk partials the same way.  So the result depends only on n_paths, not
// on which warp ran which tile.  Counters are consumed and re-zeroed by the
// warps that read them; the tile counter by the last block to exit.
template <int W>
__device__ __forceinline__ void warp_sum_strided(const double *src, uint32_t n, int lane,
                                                 double (&acc)[W]) {
#pragma unroll
  for (int v = 0; v < W; ++v) acc[v] = 0.0;
  for (uint32_t i = lane; i < n; i += 32) {
#pragma unroll
    for (int v = 0; v < W; ++v) acc[v] += __ldcg(src + size_t(i) * W + v);
  }
#pragma unroll
  for (int v = 0; v < W; ++v) acc[v] = warp_sum(acc[v]);
}

template <int W>
__device__ __noinline__ void finish_tile(const PriceArgs &a, uint64_t tile, const double (&tp)[W],
                                         int lane) {
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.control);
  uint32_t *chunk_cnt = reinterpret_cast<uint32_t *>(a.control + kChunkCountOff);
  double *chunk_part = reinterpret_cast<double *>(a.control + kChunkPartOff);
  const uint32_t chunk = uint32_t(tile / a.chunk_tiles);
  const uint64_t first = uint64_t(chunk) * a.chunk_tiles;
  const uint64_t rest = a.n_tiles - first;
  const uint32_t size = rest < a.chunk_tiles ? uint32_t(rest) : a.chunk_tiles;
  uint32_t seen = 0;
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < W; ++v) a.tile_partials[tile * W + v] = tp[v];
    // release: the partials are visible before the count that reports them
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], 1;" : "=r"(seen) : "l"(chunk_cnt + chunk) : "memory");
  }
  seen = __shfl_sync(kFull, seen, 0);
  if (seen != size - 1) return;
  // this warp completed the chunk
  __threadfence();
  double acc[W];
  warp_sum_strided<W>(a.tile_partials + first * W, size, lane, acc);
  unsigned long long done = 0;
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < W; ++v) chunk_part[size_t(chunk) * W + v] = acc[v];
    chunk_cnt[chunk] = 0;
    asm volatile("atom.release.gpu.global.add.u64 %0, [%1], 1;" : "=l"(done) : "l"(ctr + 2) : "memory");
  }
  done = __shfl_sync(kFull, done, 0);
  if (done != a.n_chunks - 1) return;
  // this warp completed the last chunk
  __threadfence();
  warp_sum_strided<W>(chunk_part, a.n_chunks, lane, acc);
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < W; ++v) a.out[v] = acc[v];
    a.out[W] = double(a.n_paths);
    ctr[2] = 0;
  }
}

}  // namespace
}  // namespace pc
