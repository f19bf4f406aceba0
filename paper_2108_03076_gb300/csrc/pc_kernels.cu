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
#include <mutex>

#include "pc_internal.h"

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

// Box-Muller on one word pair: u_a from the even word, u_b from the odd
// word; even normal r cos(2 pi u_b), odd normal r sin(2 pi u_b).  The angle
// is reduced to 2 pi u_b - pi in (-pi, pi), where cos and sin change sign.
__device__ __forceinline__ void box_muller(uint32_t xa, uint32_t xb, float &z0, float &z1) {
  const float ua = fmaf(__uint2float_rn(xa >> 8), 0x1p-24f, 0x1p-25f);
  const float r = sqrt_approx(-2.0f * logf(ua));
  const float th = fmaf(__uint2float_rn(xb >> 8), kThetaScale, kThetaOffset);
  z0 = -r * cos_approx(th);
  z1 = -r * sin_approx(th);
}

struct Rng {
  uint32_t plo, phi, stream, k0, k1;
};

__device__ __forceinline__ void block_normals(uint32_t b, const Rng &g, float *z) {
  const uint4 x = philox(make_uint4(b, g.plo, g.phi, g.stream), g.k0, g.k1);
  box_muller(x.x, x.y, z[0], z[1]);
  box_muller(x.z, x.w, z[2], z[3]);
}

#define SLOT(s) R[(s) * kBlock]

template <int D>
struct PathState {
  float w[D];   // W at the last produced date
  int f;        // last produced ordinal (frontier)
  int bsp;      // bridge stack size
};

// Normals j*D .. j*D+D-1 of bridge node j (see BridgeOp).
template <int D>
__device__ __forceinline__ void node_normals(const BridgeOp &op, const Rng &g, float *R,
                                             const Layout &lay, float (&z)[D]) {
  const uint32_t m0 = op.j * D;
  const uint32_t b0 = m0 >> 2;
  const int lane0 = int(m0 & 3u);
  float e[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int cbase = lay.off_cache + int(op.level) * 4;
  if (op.flags & BR_FROM_CACHE) {
#pragma unroll
    for (int q = 0; q < 4; ++q) e[q] = SLOT(cbase + q);
  } else {
    block_normals(b0, g, e);
  }
  const bool two = D > 1 && (op.flags & BR_TWO_BLOCKS);
  if (two) block_normals(b0 + 1, g, e + 4);
  if (op.flags & BR_STORE) {
    if (two) {
#pragma unroll
      for (int q = 0; q < 4; ++q) SLOT(cbase + q) = e[4 + q];
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) SLOT(cbase + q) = e[q];
    }
  }
  switch (lane0) {
    case 0:
#pragma unroll
      for (int i = 0; i < D; ++i) z[i] = e[i];
      break;
    case 1:
#pragma unroll
      for (int i = 0; i < D; ++i) z[i] = e[1 + i];
      break;
    case 2:
#pragma unroll
      for (int i = 0; i < D; ++i) z[i] = e[2 + i];
      break;
    default:
#pragma unroll
      for (int i = 0; i < D; ++i) z[i] = e[3 + i];
      break;
  }
}

__device__ __forceinline__ BridgeOp load_op(const BridgeOp *p) {
  const uint2 *q = reinterpret_cast<const uint2 *>(p);
  uint2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
  BridgeOp op;
  op.wl = __uint_as_float(a.x);
  op.wr = __uint_as_float(a.y);
  op.sd = __uint_as_float(b.x);
  op.j = b.y;
  op.level = uint16_t(c.x & 0xffffu);
  op.flags = uint16_t(c.x >> 16);
  op.m = uint16_t(c.y & 0xffffu);
  op.pad0 = 0;
  return op;
}

// Produce date t (= frontier + 1): bridge ops of t, then GBM into the
// window slot of t.
template <int D>
__device__ __forceinline__ void gen_date(int t, PathState<D> &ps, const ModelDev &m,
                                         const Layout &lay, const Rng &g, float *R,
                                         const float (&Bm)[D * D], const float (&S0)[D]) {
  const int k0 = __ldg(m.date_ops + t), k1 = __ldg(m.date_ops + t + 1);
  if (k0 == k1) {
    --ps.bsp;
#pragma unroll
    for (int i = 0; i < D; ++i) ps.w[i] = SLOT(lay.off_bstack + ps.bsp * D + i);
  } else {
    for (int k = k0; k < k1; ++k) {
      const BridgeOp op = load_op(m.ops + k);
      float z[D];
      node_normals<D>(op, g, R, lay, z);
      float nw[D];
      if (op.flags & BR_ROOT) {
#pragma unroll
        for (int i = 0; i < D; ++i) nw[i] = op.sd * z[i];
      } else {
        const int top = lay.off_bstack + (ps.bsp - 1) * D;
#pragma unroll
        for (int i = 0; i < D; ++i)
          nw[i] = fmaf(op.wl, ps.w[i], fmaf(op.wr, SLOT(top + i), op.sd * z[i]));
      }
      if (k + 1 < k1) {
#pragma unroll
        for (int i = 0; i < D; ++i) SLOT(lay.off_bstack + ps.bsp * D + i) = nw[i];
        ++ps.bsp;
      } else {
#pragma unroll
        for (int i = 0; i < D; ++i) ps.w[i] = nw[i];
      }
    }
  }
  const int ws = lay.off_win + (t & (lay.win - 1)) * D;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float x = __ldg(m.A + t * D + i);
#pragma unroll
    for (int k = 0; k <= i; ++k) x = fmaf(Bm[i * D + k], ps.w[k], x);
    SLOT(ws + i) = S0[i] * ex2_approx(x);
  }
  ps.f = t;
}

template <int D>
__device__ __forceinline__ void load_model_regs(const ModelDev &m, float (&Bm)[D * D],
                                                float (&S0)[D]) {
#pragma unroll
  for (int i = 0; i < D * D; ++i) Bm[i] = __ldg(m.B + i);
#pragma unroll
  for (int i = 0; i < D; ++i) S0[i] = __ldg(m.sval + m.n_hist * D + i);
}

// The payoff expression of one path per lane, all lanes of the warp in step.
template <int D>
__device__ float eval_path(const uint4 *P, float *R, const PriceArgs &a, const Rng &g,
                           bool live, const float (&Bm)[D * D], const float (&S0)[D]) {
  const ModelDev &m = a.m;
  const Layout &lay = a.lay;
  PathState<D> ps;
#pragma unroll
  for (int i = 0; i < D; ++i) ps.w[i] = 0.f;
  ps.f = 0;
  ps.bsp = 0;
  const int t_now = m.t_now;
  int pc = 0, sp = 0, t0 = 0;
  float tos = 0.f;
#define PUSH(v)         \
  do {                  \
    SLOT(sp) = tos;     \
    ++sp;               \
    tos = (v);          \
  } while (0)
#define BINF(expr)                  \
  {                                 \
    const float b_ = tos;           \
    const float a_ = SLOT(sp - 1);  \
    --sp;                           \
    tos = (expr);                   \
    ++pc;                           \
    break;                          \
  }
#define BINI(expr)                                  \
  {                                                 \
    const int b_ = __float_as_int(tos);             \
    const int a_ = __float_as_int(SLOT(sp - 1));    \
    --sp;                                           \
    tos = __int_as_float(expr);                     \
    ++pc;                                           \
    break;                                          \
  }
#define IMM(expr)                            \
  {                                          \
    const float k_ = __uint_as_float(I.y);   \
    const float x_ = tos;                    \
    tos = (expr);                            \
    ++pc;                                    \
    break;                                   \
  }
  for (;;) {
    const uint4 I = P[pc];
    switch (I.x & 0xffu) {
      case X_CONST: PUSH(__uint_as_float(I.y)); ++pc; break;
      case X_MODEL:
      case X_MODEL_MULK:
      case X_MODEL_DIVK: {
        int o = int(I.y) + t0 - t_now;
        const int l = int(I.x >> 8) & 7;
        float v;
        if (o > 0) {
          if (o > m.n) {  // unreachable after the load-time analysis; keep memory safe
            atomicOr(a.status, 1);
            o = m.n;
          }
          while (ps.f < o) gen_date<D>(ps.f + 1, ps, m, lay, g, R, Bm, S0);
          v = SLOT(lay.off_win + (o & (lay.win - 1)) * D + (l < D ? l : 0));
        } else {
          if (o < -m.n_hist) {
            atomicOr(a.status, 1);
            o = -m.n_hist;
          }
          v = __ldg(m.sval + (o + m.n_hist) * D + (l < D ? l : 0));
        }
        const uint32_t op = I.x & 0xffu;
        if (op == X_MODEL_MULK) v *= __uint_as_float(I.z);
        else if (op == X_MODEL_DIVK) v = __fdiv_rn(v, __uint_as_float(I.z));
        PUSH(v);
        ++pc;
        break;
      }
      case X_PAYOFF: {
        int o = int(I.y) + t0 - t_now;
        if (o > m.n || o < -m.n_hist) {
          atomicOr(a.status, 1);
          o = 0;
        }
        float v = __ldg(m.disc + o + m.n_hist);
        if (I.x >> 8) v = -v;
        PUSH(v);
        ++pc;
        break;
      }
      case X_TIME: PUSH(__int_as_float(int(I.y) + t0)); ++pc; break;
      case X_NOW: PUSH(__int_as_float(t_now)); ++pc; break;
      case X_NEGF: tos = -tos; ++pc; break;
      case X_NOT: tos = __int_as_float(__float_as_int(tos) ^ 1); ++pc; break;
      case X_ADDF: BINF(a_ + b_)
      case X_SUBF: BINF(a_ - b_)
      case X_MULF: BINF(a_ * b_)
      case X_DIVF: BINF(__fdiv_rn(a_, b_))
      case X_MAXF: BINF(fmaxf(a_, b_))
      case X_MINF: BINF(fminf(a_, b_))
      case X_LTF: BINF(__int_as_float(int(a_ < b_)))
      case X_LEF: BINF(__int_as_float(int(a_ <= b_)))
      case X_EQF: BINF(__int_as_float(int(a_ == b_)))
      case X_ADDI: BINI(a_ + b_)
      case X_SUBI: BINI(a_ > b_ ? a_ - b_ : 0)
      case X_MULI: BINI(a_ * b_)
      case X_MAXI: BINI(a_ > b_ ? a_ : b_)
      case X_MINI: BINI(a_ < b_ ? a_ : b_)
      case X_LTI: BINI(int(a_ < b_))
      case X_LEI: BINI(int(a_ <= b_))
      case X_EQI: BINI(int(a_ == b_))
      case X_AND: BINI(a_ & b_)
      case X_OR: BINI(a_ | b_)
      case X_ADDFK: IMM(x_ + k_)
      case X_SUBFK: IMM(x_ - k_)
      case X_MULFK: IMM(x_ * k_)
      case X_DIVFK: IMM(__fdiv_rn(x_, k_))
      case X_MAXFK: IMM(fmaxf(x_, k_))
      case X_MINFK: IMM(fminf(x_, k_))
      case X_LTFK: IMM(__int_as_float(int(x_ < k_)))
      case X_LEFK: IMM(__int_as_float(int(x_ <= k_)))
      case X_EQFK: IMM(__int_as_float(int(x_ == k_)))
      case X_RSUBFK: IMM(k_ - x_)
      case X_RDIVFK: IMM(__fdiv_rn(k_, x_))
      case X_RLTFK: IMM(__int_as_float(int(k_ < x_)))
      case X_RLEFK: IMM(__int_as_float(int(k_ <= x_)))
      case X_IF: {
        const bool c = __float_as_int(tos) != 0;
        if (__any_sync(kFull, live && c)) {
          ++pc;
        } else {
          PUSH(0.f);
          pc = int(I.z);
        }
        break;
      }
      case X_ELSE: {
        const bool c = __float_as_int(SLOT(sp - 1)) != 0;
        if (__any_sync(kFull, live && !c)) {
          ++pc;
        } else {
          PUSH(0.f);
          pc = int(I.z);
        }
        break;
      }
      case X_SEL: {
        const float th = SLOT(sp - 1);
        const int c = __float_as_int(SLOT(sp - 2));
        sp -= 2;
        tos = c ? th : tos;
        ++pc;
        break;
      }
      case X_LOOP: {
        const int F = int(I.x >> 8);
        SLOT(F + LF_K) = __int_as_float(0);
        SLOT(F + LF_T0) = __int_as_float(t0);
        SLOT(F + LF_DONE) = __int_as_float(live ? 0 : 1);
        SLOT(F + LF_RES) = 0.f;
        ++pc;
        break;
      }
      case X_LTEST: {
        const int F = int(I.x >> 8);
        const int c = __float_as_int(tos);
        --sp;
        tos = SLOT(sp);
        const int nw = (c != 0) && (__float_as_int(SLOT(F + LF_DONE)) == 0);
        SLOT(F + LF_NEWLY) = __int_as_float(nw);
        pc = __any_sync(kFull, nw) ? pc + 1 : int(I.z);
        break;
      }
      case X_LLATCH: {
        const int F = int(I.x >> 8);
        const float v = tos;
        --sp;
        tos = SLOT(sp);
        if (__float_as_int(SLOT(F + LF_NEWLY))) {
          SLOT(F + LF_RES) = v;
          SLOT(F + LF_DONE) = __int_as_float(1);
        }
        ++pc;
        break;
      }
      case X_LNEXT: {
        const int F = int(I.x >> 8);
        const int t0e = __float_as_int(SLOT(F + LF_T0));
        if (__all_sync(kFull, __float_as_int(SLOT(F + LF_DONE)) != 0)) {
          t0 = t0e;
          PUSH(SLOT(F + LF_RES));
          pc = int(I.w);
        } else {
          int k = __float_as_int(SLOT(F + LF_K));
          if (k == int(I.y)) {
            t0 = t0e + k;
            ++pc;
          } else {
            ++k;
            SLOT(F + LF_K) = __int_as_float(k);
            t0 = t0e + k;
            pc = int(I.z);
          }
        }
        break;
      }
      case X_LEND: {
        const int F = int(I.x >> 8);
        if (__float_as_int(SLOT(F + LF_DONE))) tos = SLOT(F + LF_RES);
        t0 = __float_as_int(SLOT(F + LF_T0));
        ++pc;
        break;
      }
      default:
        return tos;
    }
  }
#undef PUSH
#undef BINF
#undef BINI
#undef IMM
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Fixed-order sum of the tile partials by the last block to finish: thread t
// adds tiles t, t + kBlock, ... in order, then a fixed tree over the block.
__device__ void final_reduce(const PriceArgs &a, double *red) {
  for (int v = 0; v < a.width; ++v) {
    double s = 0.0;
    for (uint64_t t = threadIdx.x; t < a.n_tiles; t += kBlock)
      s += a.tile_partials[t * a.width + v];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kBlock / 2; h > 0; h >>= 1) {
      if (int(threadIdx.x) < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) a.out[v] = red[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.out[a.width] = double(a.n_paths);
}

// Tiles of kTilePaths consecutive paths are handed to warps through an
// atomic counter; each tile's (sum, sum of squares) is reduced in FP64 over
// the warp in a fixed shuffle order and stored at the tile's index, so the
// result does not depend on which warp ran which tile.  The last block to
// finish sums the tiles in index order and resets the counters.
template <int D, bool WRITE>
__global__ void __launch_bounds__(kBlock) price_kernel(const PriceArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ double red[kBlock];
  __shared__ int last_block;
  uint4 *P = reinterpret_cast<uint4 *>(smem);
  const uint4 *src = reinterpret_cast<const uint4 *>(a.prog);
  for (int i = threadIdx.x; i < a.n_insn; i += kBlock) P[i] = src[i];
  __syncthreads();
  float *R = reinterpret_cast<float *>(smem + a.n_insn * 4) + threadIdx.x;
  float Bm[D * D], S0[D];
  load_model_regs<D>(a.m, Bm, S0);
  const int lane = threadIdx.x & 31;
  Rng g;
  g.stream = a.stream;
  g.k0 = a.key0;
  g.k1 = a.key1;
  for (;;) {
    unsigned long long tile = 0;
    if (lane == 0) tile = atomicAdd(a.counters, 1ull);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= a.n_tiles) break;
    double s = 0.0, s2 = 0.0;
#pragma unroll 1
    for (int q = 0; q < kPathsPerLane; ++q) {
      const uint64_t idx = tile * kTilePaths + uint64_t(q) * 32 + lane;
      const bool live = idx < a.n_paths;
      const uint64_t p = a.path_offset + idx;
      g.plo = uint32_t(p);
      g.phi = uint32_t(p >> 32);
      const float x = eval_path<D>(P, R, a, g, live, Bm, S0);
      if (live) {
        const double xd = double(x);
        s += xd;
        s2 = fma(xd, xd, s2);
        if (WRITE) a.out_paths[idx] = x;
      }
    }
    s = warp_sum(s);
    s2 = warp_sum(s2);
    if (lane == 0) {
      a.tile_partials[2 * tile] = s;
      a.tile_partials[2 * tile + 1] = s2;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_block = atomicAdd(a.counters + 1, 1ull) == gridDim.x - 1;
  __syncthreads();
  if (last_block) {
    __threadfence();
    final_reduce(a, red);
    if (threadIdx.x == 0) {
      a.counters[0] = 0;
      a.counters[1] = 0;
    }
  }
}

__global__ void debug_philox_kernel(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                    size_t n) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = reinterpret_cast<const uint4 *>(ctr)[i];
  reinterpret_cast<uint4 *>(out)[i] = philox(c, k0, k1);
}

template <int D>
__global__ void __launch_bounds__(kBlock) debug_paths_kernel(const ModelDev m, const Layout lay,
                                                             uint64_t n_paths, uint64_t offset,
                                                             uint32_t k0, uint32_t k1,
                                                             uint32_t stream, float *out) {
  extern __shared__ __align__(16) uint32_t smem[];
  float *R = reinterpret_cast<float *>(smem) + threadIdx.x;
  const uint64_t i = uint64_t(blockIdx.x) * kBlock + threadIdx.x;
  if (i >= n_paths) return;
  float Bm[D * D], S0[D];
  load_model_regs<D>(m, Bm, S0);
  Rng g{uint32_t(offset + i), uint32_t((offset + i) >> 32), stream, k0, k1};
  PathState<D> ps;
#pragma unroll
  for (int l = 0; l < D; ++l) ps.w[l] = 0.f;
  ps.f = 0;
  ps.bsp = 0;
  const size_t row = size_t(m.n) + 1;
  for (int l = 0; l < D; ++l) out[(i * D + l) * row] = S0[l];
  for (int t = 1; t <= m.n; ++t) {
    gen_date<D>(t, ps, m, lay, g, R, Bm, S0);
    const int ws = lay.off_win + (t & (lay.win - 1)) * D;
    for (int l = 0; l < D; ++l) out[(i * D + l) * row + t] = SLOT(ws + l);
  }
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

}  // namespace

cudaError_t launch_price(const PriceArgs &a, int grid, size_t smem, cudaStream_t s) {
  const bool w = a.out_paths != nullptr;
#define LAUNCH(DD, WW)                                                             \
  do {                                                                             \
    auto k = price_kernel<DD, WW>;                                                 \
    cudaError_t e = set_smem(k, smem);                                             \
    if (e != cudaSuccess) return e;                                                \
    k<<<grid, kBlock, smem, s>>>(a);                                               \
    return cudaGetLastError();                                                     \
  } while (0)
  switch (a.m.d) {
    case 1: if (w) LAUNCH(1, true); else LAUNCH(1, false);
    case 2: if (w) LAUNCH(2, true); else LAUNCH(2, false);
    case 3: if (w) LAUNCH(3, true); else LAUNCH(3, false);
    case 4: if (w) LAUNCH(4, true); else LAUNCH(4, false);
    default: return cudaErrorInvalidValue;
  }
#undef LAUNCH
}

int price_blocks_per_sm(int d, size_t smem, bool greeks) {
  (void)greeks;
  int nb = 0;
  cudaError_t e = cudaSuccess;
  switch (d) {
    case 1: set_smem(price_kernel<1, false>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<1, false>, kBlock, smem); break;
    case 2: set_smem(price_kernel<2, false>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<2, false>, kBlock, smem); break;
    case 3: set_smem(price_kernel<3, false>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<3, false>, kBlock, smem); break;
    case 4: set_smem(price_kernel<4, false>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<4, false>, kBlock, smem); break;
    default: return 0;
  }
  return e == cudaSuccess ? nb : 0;
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
  const size_t smem = size_t(lay.words) * kBlock * 4;
  const unsigned grid = unsigned((n_paths + kBlock - 1) / kBlock);
  if (grid == 0) return cudaSuccess;
#define DLAUNCH(DD)                                                                 \
  do {                                                                              \
    auto k = debug_paths_kernel<DD>;                                                \
    cudaError_t e = set_smem(k, smem);                                              \
    if (e != cudaSuccess) return e;                                                 \
    k<<<grid, kBlock, smem, s>>>(m, lay, n_paths, offset, k0, k1, stream, out);     \
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

// Scratch of pc_price_noalloc: work counters in the first 256 bytes, then
// one (sum, sum of squares) pair per tile of kTilePaths paths for up to
// PC_NOALLOC_MAX_PATHS paths.  Zero-initialised when the module loads;
// each call clears the counters again before its launch.
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

cudaError_t launch_greeks(const PriceArgs &, int, size_t, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace pc
