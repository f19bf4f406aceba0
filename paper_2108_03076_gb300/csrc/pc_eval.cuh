// pc_eval.cuh -- the warp-uniform payoff interpreter (eval_path), shared by
// the pricing, portfolio and control-variate kernels.
#pragma once

#include "pc_device.cuh"

namespace pc {
namespace {

// The payoff expression of two paths per lane, all lanes of the warp in step.
// The next instruction is fetched while the current one executes; jumps
// fetch their target.  `frontier` (optional) receives the last generated
// date ordinal: the window holds the simulated dates up to it.
template <int D, bool GW = false>
__device__ float2 eval_path(const uint4 *P, const float *pool, float2 *R, const PriceArgs &a,
                            const Rng2 &g, bool live0, bool live1, const float (&Bm)[D * D],
                            const float (&S0)[D], int *frontier = nullptr) {
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
    while (ps.f < o) gen_date<D, false, GW>(ps.f + 1, ps, m, lay, g, R, Bm, S0);
  };
  auto read = [&](int o, int l) -> float2 {
    l = l < D ? l : 0;
    if (o > 0) return win_load<GW>(R, lay, (o & (lay.win - 1)) * D + l);
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
        PUSH((fused_value<D, GW>(I, o, pool, R, m, lay)));
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
          const float2 c = fused_value<D, GW>(Dsc, o, pool, R, m, lay);
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
        if (frontier) *frontier = ps.f;
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

}  // namespace
}  // namespace pc
