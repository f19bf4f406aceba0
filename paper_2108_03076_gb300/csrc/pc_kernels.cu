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

#include "pc_device.cuh"

namespace pc {

namespace {

// The payoff expression of two paths per lane, all lanes of the warp in step.
// The next instruction is fetched while the current one executes; jumps
// fetch their target.
template <int D>
__device__ float2 eval_path(const uint4 *P, const float *pool, float2 *R, const PriceArgs &a,
                            const Rng2 &g, bool live0, bool live1, const float (&Bm)[D * D],
                            const float (&S0)[D]) {
  const ModelDev &m = a.m;
  const Layout &lay = a.lay;
  PathState<D> ps;
#pragma unroll
  for (int i = 0; i < D; ++i) ps.w[i] = make_float2(0.f, 0.f);
  ps.f = 0;
  ps.bsp = 0;
  const int t_now = m.t_now;
  int pc = 0, sp = 0, t0 = 0;
  float2 tos = make_float2(0.f, 0.f);
  // frontier advance to ordinal o (clamped into the grid if the load-time
  // analysis were ever wrong)
  auto ensure = [&](int &o) {
    if (o > m.n || o < -m.n_hist) {
      atomicOr(a.status, 1);
      o = o > m.n ? m.n : -m.n_hist;
    }
    while (ps.f < o) gen_date<D>(ps.f + 1, ps, m, lay, g, R, Bm, S0);
  };
  auto read = [&](int o, int l) -> float2 {
    l = l < D ? l : 0;
    if (o > 0) return SL(lay.off_win + (o & (lay.win - 1)) * D + l);
    const float v = __ldg(m.sval + (o + m.n_hist) * D + l);
    return make_float2(v, v);
  };
#define NEXT      \
  {               \
    ++pc;         \
    I = In;       \
    break;        \
  }
#define JUMP(t)   \
  {               \
    pc = (t);     \
    I = P[pc];    \
    break;        \
  }
#define PUSH(v)        \
  do {                 \
    SL(sp) = tos;      \
    ++sp;              \
    tos = (v);         \
  } while (0)
#define BINF(expr)                                                         \
  {                                                                        \
    const float2 B_ = tos, A_ = SL(sp - 1);                                \
    --sp;                                                                  \
    { const float a_ = A_.x, b_ = B_.x; tos.x = (expr); }                  \
    { const float a_ = A_.y, b_ = B_.y; tos.y = (expr); }                  \
    NEXT                                                                   \
  }
#define BINI(expr)                                                         \
  {                                                                        \
    const float2 B_ = tos, A_ = SL(sp - 1);                                \
    --sp;                                                                  \
    { const int a_ = bits(A_.x), b_ = bits(B_.x); tos.x = fl(expr); }     \
    { const int a_ = bits(A_.y), b_ = bits(B_.y); tos.y = fl(expr); }     \
    NEXT                                                                   \
  }
#define IMM(expr)                                                          \
  {                                                                        \
    const float k_ = __uint_as_float(I.y);                                 \
    { const float x_ = tos.x; tos.x = (expr); }                            \
    { const float x_ = tos.y; tos.y = (expr); }                            \
    NEXT                                                                   \
  }
  uint4 I = P[0];
  for (;;) {
    const uint4 In = P[pc + 1];
    switch (I.x & 0xffu) {
      case X_CONST: PUSH(make_float2(__uint_as_float(I.y), __uint_as_float(I.y))); NEXT
      case X_MODEL:
      case X_MODEL_MULK:
      case X_MODEL_DIVK: {
        int o = int(I.y) + t0 - t_now;
        ensure(o);
        float2 v = read(o, int(I.x >> 8) & 3);
        const uint32_t op = I.x & 0xffu;
        const float k = __uint_as_float(I.z);
        if (op == X_MODEL_MULK) v = make_float2(v.x * k, v.y * k);
        else if (op == X_MODEL_DIVK) v = make_float2(__fdiv_rn(v.x, k), __fdiv_rn(v.y, k));
        PUSH(v);
        NEXT
      }
      case X_LRED:
      case X_LANY: {
        int o = int(I.y) + t0 - t_now;
        ensure(o);
        PUSH(fused_value<D>(I, o, pool, R, m, lay));
        NEXT
      }
      case X_PAYOFF: {
        int o = int(I.y) + t0 - t_now;
        if (o > m.n || o < -m.n_hist) {
          atomicOr(a.status, 1);
          o = 0;
        }
        float v = __uint_as_float(I.z) * __ldg(m.disc + o + m.n_hist);
        if (I.x >> 8) v = -v;
        PUSH(make_float2(v, v));
        NEXT
      }
      case X_TIME: PUSH(fl2(int(I.y) + t0, int(I.y) + t0)); NEXT
      case X_NOW: PUSH(fl2(t_now, t_now)); NEXT
      case X_NEGF: tos = make_float2(-tos.x, -tos.y); NEXT
      case X_NOT: tos = fl2(bits(tos.x) ^ 1, bits(tos.y) ^ 1); NEXT
      case X_ADDF: BINF(a_ + b_)
      case X_SUBF: BINF(a_ - b_)
      case X_MULF: BINF(a_ * b_)
      case X_DIVF: BINF(__fdiv_rn(a_, b_))
      case X_MAXF: BINF(fmaxf(a_, b_))
      case X_MINF: BINF(fminf(a_, b_))
      case X_LTF: BINF(fl(int(a_ < b_)))
      case X_LEF: BINF(fl(int(a_ <= b_)))
      case X_EQF: BINF(fl(int(a_ == b_)))
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
      case X_LTFK: IMM(fl(int(x_ < k_)))
      case X_LEFK: IMM(fl(int(x_ <= k_)))
      case X_EQFK: IMM(fl(int(x_ == k_)))
      case X_RSUBFK: IMM(k_ - x_)
      case X_RDIVFK: IMM(__fdiv_rn(k_, x_))
      case X_RLTFK: IMM(fl(int(k_ < x_)))
      case X_RLEFK: IMM(fl(int(k_ <= x_)))
      case X_IF: {
        const bool c0 = bits(tos.x) != 0, c1 = bits(tos.y) != 0;
        if (__any_sync(kFull, (live0 && c0) || (live1 && c1))) NEXT
        PUSH(make_float2(0.f, 0.f));
        JUMP(int(I.z))
      }
      case X_ELSE: {
        const float2 c = SL(sp - 1);
        const bool c0 = bits(c.x) != 0, c1 = bits(c.y) != 0;
        if (__any_sync(kFull, (live0 && !c0) || (live1 && !c1))) NEXT
        PUSH(make_float2(0.f, 0.f));
        JUMP(int(I.z))
      }
      case X_SEL: {
        const float2 th = SL(sp - 1), c = SL(sp - 2);
        sp -= 2;
        tos = make_float2(bits(c.x) ? th.x : tos.x, bits(c.y) ? th.y : tos.y);
        NEXT
      }
      case X_LOOP: {
        const int F = int(I.x >> 8);
        SL(F + LF_K) = fl2(0, 0);
        SL(F + LF_T0) = fl2(t0, t0);
        SL(F + LF_DONE) = fl2(live0 ? 0 : 1, live1 ? 0 : 1);
        SL(F + LF_RES) = make_float2(0.f, 0.f);
        NEXT
      }
      case X_LOOPANY: {
        const int F = int((I.x >> 8) & 0xffu);
        const float lit = pool[I.x >> 16];
        const uint4 Dsc = In;  // the condition descriptor
        bool d0 = !live0, d1 = !live1;
        float r0 = 0.f, r1 = 0.f;
        const int n = int(I.y);
        bool all = false;
        for (int k = 0;; ++k) {
          int o = int(Dsc.y) + t0 + k - t_now;
          ensure(o);
          const float2 c = fused_value<D>(Dsc, o, pool, R, m, lay);
          if (bits(c.x) && !d0) { d0 = true; r0 = lit; }
          if (bits(c.y) && !d1) { d1 = true; r1 = lit; }
          all = __all_sync(kFull, d0 && d1);
          if (all || k == n) break;
        }
        if (all) {
          PUSH(make_float2(r0, r1));
          JUMP(int(I.w))
        }
        SL(F + LF_T0) = fl2(t0, t0);
        SL(F + LF_DONE) = fl2(d0, d1);
        SL(F + LF_RES) = make_float2(r0, r1);
        t0 += n;
        JUMP(pc + 2)
      }
      case X_LTEST: {
        const int F = int(I.x >> 8);
        const float2 c = tos;
        --sp;
        tos = SL(sp);
        const float2 d = SL(F + LF_DONE);
        const int n0 = bits(c.x) != 0 && bits(d.x) == 0, n1 = bits(c.y) != 0 && bits(d.y) == 0;
        SL(F + LF_NEWLY) = fl2(n0, n1);
        if (__any_sync(kFull, n0 | n1)) NEXT
        JUMP(int(I.z))
      }
      case X_LLATCH: {
        const int F = int(I.x >> 8);
        const float2 v = tos;
        --sp;
        tos = SL(sp);
        const float2 nw = SL(F + LF_NEWLY);
        if (bits(nw.x) | bits(nw.y)) {
          const float2 r = SL(F + LF_RES), d = SL(F + LF_DONE);
          SL(F + LF_RES) = make_float2(bits(nw.x) ? v.x : r.x, bits(nw.y) ? v.y : r.y);
          SL(F + LF_DONE) = fl2(bits(d.x) | bits(nw.x), bits(d.y) | bits(nw.y));
        }
        NEXT
      }
      case X_LSTEPK:
      case X_LNEXT: {
        const bool step = (I.x & 0xffu) == X_LSTEPK;
        const int F = step ? int((I.x >> 8) & 0xffu) : int(I.x >> 8);
        float2 d = SL(F + LF_DONE);
        if (step) {  // latch the literal on lanes whose test newly holds
          const float2 c = tos;
          --sp;
          tos = SL(sp);
          const int n0 = bits(c.x) != 0 && bits(d.x) == 0, n1 = bits(c.y) != 0 && bits(d.y) == 0;
          if (n0 | n1) {
            const float lit = pool[I.x >> 16];
            const float2 r = SL(F + LF_RES);
            SL(F + LF_RES) = make_float2(n0 ? lit : r.x, n1 ? lit : r.y);
            d = fl2(bits(d.x) | n0, bits(d.y) | n1);
            SL(F + LF_DONE) = d;
          }
        }
        const int t0e = bits(SL(F + LF_T0).x);
        if (__all_sync(kFull, (bits(d.x) & bits(d.y)) != 0)) {
          t0 = t0e;
          PUSH(SL(F + LF_RES));
          JUMP(int(I.w))
        }
        int k = bits(SL(F + LF_K).x);
        if (k == int(I.y)) {
          t0 = t0e + k;
          NEXT
        }
        ++k;
        SL(F + LF_K) = fl2(k, k);
        t0 = t0e + k;
        JUMP(int(I.z))
      }
      case X_LEND: {
        const int F = int(I.x >> 8);
        const float2 d = SL(F + LF_DONE), r = SL(F + LF_RES);
        tos = make_float2(bits(d.x) ? r.x : tos.x, bits(d.y) ? r.y : tos.y);
        t0 = bits(SL(F + LF_T0).x);
        NEXT
      }
      default:
        return tos;
    }
  }
#undef NEXT
#undef JUMP
#undef PUSH
#undef BINF
#undef BINI
#undef IMM
}

// Tiles of kTilePaths consecutive paths (two per lane: tile*64 + lane and
// tile*64 + 32 + lane) are handed to warps through an atomic counter.
template <int D, bool WRITE>
__global__ void __launch_bounds__(kBlock) price_kernel(const PriceArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int last_block;
  uint4 *P = reinterpret_cast<uint4 *>(smem);
  const int prog_words = a.n_insn * 4 + a.n_pool;
  const uint32_t *src = reinterpret_cast<const uint32_t *>(a.prog);
  for (int i = threadIdx.x; i < prog_words; i += blockDim.x) smem[i] = src[i];
  __syncthreads();
  const float *pool = reinterpret_cast<const float *>(smem + a.n_insn * 4);
  float2 *R = reinterpret_cast<float2 *>(smem + prog_words) + threadIdx.x;
  float Bm[D * D], S0[D];
  load_model_regs<D>(a.m, Bm, S0);
  const int lane = threadIdx.x & 31;
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.control);
  Rng2 g;
  g.stream = a.stream;
  g.k0 = a.key0;
  g.k1 = a.key1;
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
    const float2 x = eval_path<D>(P, pool, R, a, g, live0, live1, Bm, S0);
    double tp[2] = {0.0, 0.0};
    if (live0) {
      const double xd = double(x.x);
      tp[0] += xd;
      tp[1] = fma(xd, xd, tp[1]);
      if (WRITE) a.out_paths[i0] = x.x;
    }
    if (live1) {
      const double xd = double(x.y);
      tp[0] += xd;
      tp[1] = fma(xd, xd, tp[1]);
      if (WRITE) a.out_paths[i1] = x.y;
    }
    tp[0] = warp_sum(tp[0]);
    tp[1] = warp_sum(tp[1]);
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

// Portfolio kernel.  Warps take work units (a contract and a run of its
// tiles) from the group's counter in the order of the unit array.  When a
// warp's unit belongs to another contract than its previous one, the warp
// copies that contract's arguments, program and constant pool into its own
// slot of shared memory.  The tiles run as in price_kernel and finish into
// the contract's own reduction scratch, so each contract's sums are those of
// a single-contract launch.
template <int D>
__global__ void __launch_bounds__(kBlock) batch_kernel(const BatchArgs b) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *slot = smem + (b.slot_bytes / 4) * warp;
  float2 *R = reinterpret_cast<float2 *>(smem + (b.slot_bytes / 4) * (blockDim.x >> 5)) + threadIdx.x;
  const PriceArgs &a = *reinterpret_cast<const PriceArgs *>(slot);
  const uint4 *P = reinterpret_cast<const uint4 *>(slot + kBatchArgsBytes / 4);
  float Bm[D * D], S0[D];
  Rng2 g;
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
      const int n_words = a.n_insn * 4 + a.n_pool;
      const uint32_t *code = reinterpret_cast<const uint32_t *>(a.prog);
      for (int i = lane; i < n_words; i += 32) slot[kBatchArgsBytes / 4 + i] = __ldg(code + i);
      __syncwarp();
      cur = U.item;
    }
    const float *pool = reinterpret_cast<const float *>(P + a.n_insn);
    load_model_regs<D>(a.m, Bm, S0);
    g.stream = a.stream;
    g.k0 = a.key0;
    g.k1 = a.key1;
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
      double tp[2] = {0.0, 0.0};
      if (live0) {
        const double xd = double(x.x);
        tp[0] += xd;
        tp[1] = fma(xd, xd, tp[1]);
      }
      if (live1) {
        const double xd = double(x.y);
        tp[0] += xd;
        tp[1] = fma(xd, xd, tp[1]);
      }
      tp[0] = warp_sum(tp[0]);
      tp[1] = warp_sum(tp[1]);
      finish_tile<2>(a, tile, tp, lane);
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

// Thread t generates paths offset + 2t and offset + 2t + 1 with the pricing
// kernel's generator and writes every date of both.
template <int D>
__global__ void __launch_bounds__(kBlock) debug_paths_kernel(const ModelDev m, const Layout lay,
                                                             uint64_t n_paths, uint64_t offset,
                                                             uint32_t k0, uint32_t k1,
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
  g.k0 = k0;
  g.k1 = k1;
  PathState<D> ps;
#pragma unroll
  for (int l = 0; l < D; ++l) ps.w[l] = make_float2(0.f, 0.f);
  ps.f = 0;
  ps.bsp = 0;
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
  const bool w = a.out_paths != nullptr;
#define LAUNCH(DD, WW)                                                             \
  do {                                                                             \
    auto k = price_kernel<DD, WW>;                                                 \
    cudaError_t e = set_smem(k, smem);                                             \
    if (e != cudaSuccess) return e;                                                \
    k<<<grid, block, smem, s>>>(a);                                                \
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

int price_blocks_per_sm(int d, int block, size_t smem, bool greeks) {
  (void)greeks;
  int nb = 0;
  cudaError_t e = cudaSuccess;
  switch (d) {
    case 1: set_smem(price_kernel<1, false>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<1, false>, block, smem); break;
    case 2: set_smem(price_kernel<2, false>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<2, false>, block, smem); break;
    case 3: set_smem(price_kernel<3, false>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<3, false>, block, smem); break;
    case 4: set_smem(price_kernel<4, false>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, price_kernel<4, false>, block, smem); break;
    default: return 0;
  }
  return e == cudaSuccess ? nb : 0;
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
  if (grid == 0) return cudaSuccess;
#define DLAUNCH(DD)                                                                 \
  do {                                                                              \
    auto k = debug_paths_kernel<DD>;                                                \
    cudaError_t e = set_smem(k, smem);                                              \
    if (e != cudaSuccess) return e;                                                 \
    k<<<grid, block, smem, s>>>(m, lay, n_paths, offset, k0, k1, stream, out);      \
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
