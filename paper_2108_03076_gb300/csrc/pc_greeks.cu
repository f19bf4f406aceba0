// pc_greeks.cu -- pathwise sensitivities of the Monte Carlo price.
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
#include <cstdint>

#include "pc_device.cuh"
#include "pc_internal.h"

namespace pc {
namespace {

struct TV {
  float2 v, a, b;  // value, d/dS0_g, d/dsigma_g (two paths each)
};

__device__ __forceinline__ TV tv(float2 v) { return {v, make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 add2(float2 p, float2 q) { return f2(p.x + q.x, p.y + q.y); }
__device__ __forceinline__ float2 sub2(float2 p, float2 q) { return f2(p.x - q.x, p.y - q.y); }
__device__ __forceinline__ float2 mul2(float2 p, float2 q) { return f2(p.x * q.x, p.y * q.y); }
__device__ __forceinline__ float2 scl2(float2 p, float k) { return f2(p.x * k, p.y * k); }
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
    const float st = sig_g * __ldg(m.tau + o);
    return {s, scl2(s, 1.0f / S0[l]), f2(s.x * (x.x - st), s.y * (x.y - st))};
  }
  const float v = __ldg(m.sval + (o + m.n_hist) * D + l);
  TV r = tv(f2(v, v));
  if (o == 0 && l == g) r.a = f2(1.f, 1.f);
  return r;
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
  const ModelDev &m = a.m;
  const Layout &lay = a.lay;
  PathState<D> ps;
#pragma unroll
  for (int i = 0; i < D; ++i) ps.w[i] = f2(0.f, 0.f);
  ps.f = 0;
  ps.bsp = 0;
  const int t_now = m.t_now;
  int pc = 0, sp = 0, t0 = 0;
  TV tos = tv(f2(0.f, 0.f));
  auto ensure = [&](int &o) {
    if (o > m.n || o < -m.n_hist) {
      atomicOr(a.status, 1);
      o = o > m.n ? m.n : -m.n_hist;
    }
    while (ps.f < o) gen_date<D, true>(ps.f + 1, ps, m, lay, g, R, Bm, S0, Lm);
  };
  auto push = [&](const TV &v) {
    stv(R, sp, tos);
    ++sp;
    tos = v;
  };
  auto pop = [&]() {
    const TV v = tos;
    --sp;
    tos = ldv(R, sp);
    return v;
  };
  // frame slot helpers (value part of logical slot F + j)
  auto fget = [&](int F, int j) { return SL(3 * (F + j)); };
  auto fset = [&](int F, int j, float2 v) { SL(3 * (F + j)) = v; };
  for (;;) {
    const uint4 I = P[pc];
    const uint32_t op = I.x & 0xffu;
    const float kk = __uint_as_float(I.y);
    switch (op) {
      case X_CONST: push(tv(f2(kk, kk))); ++pc; break;
      case X_MODEL:
      case X_MODEL_MULK:
      case X_MODEL_DIVK: {
        int o = int(I.y) + t0 - t_now;
        ensure(o);
        TV v = model_read<D>(o, int(I.x >> 8) & 3, gl, R, m, lay, S0, sig_g);
        const float k = __uint_as_float(I.z);
        if (op == X_MODEL_MULK) v = {scl2(v.v, k), scl2(v.a, k), scl2(v.b, k)};
        else if (op == X_MODEL_DIVK)
          v = {f2(__fdiv_rn(v.v.x, k), __fdiv_rn(v.v.y, k)), f2(__fdiv_rn(v.a.x, k), __fdiv_rn(v.a.y, k)),
               f2(__fdiv_rn(v.b.x, k), __fdiv_rn(v.b.y, k))};
        push(v);
        ++pc;
        break;
      }
      case X_LRED:
      case X_LANY: {
        int o = int(I.y) + t0 - t_now;
        ensure(o);
        push(fused_tv<D>(I, o, pool, R, m, lay, S0, gl, sig_g));
        ++pc;
        break;
      }
      case X_PAYOFF: {
        int o = int(I.y) + t0 - t_now;
        if (o > m.n || o < -m.n_hist) {
          atomicOr(a.status, 1);
          o = 0;
        }
        float v = __uint_as_float(I.z) * __ldg(m.disc + o + m.n_hist);
        if (I.x >> 8) v = -v;
        push(tv(f2(v, v)));
        ++pc;
        break;
      }
      case X_TIME: push(tv(fl2(int(I.y) + t0, int(I.y) + t0))); ++pc; break;
      case X_NOW: push(tv(fl2(t_now, t_now))); ++pc; break;
      case X_NEGF: tos = {neg2(tos.v), neg2(tos.a), neg2(tos.b)}; ++pc; break;
      case X_NOT: tos = tv(fl2(bits(tos.v.x) ^ 1, bits(tos.v.y) ^ 1)); ++pc; break;
      case X_ADDF: case X_SUBF: case X_MULF: case X_DIVF: case X_MAXF: case X_MINF: {
        const TV y = pop(), x = tos;
        TV r;
        if (op == X_ADDF) r = {add2(x.v, y.v), add2(x.a, y.a), add2(x.b, y.b)};
        else if (op == X_SUBF) r = {sub2(x.v, y.v), sub2(x.a, y.a), sub2(x.b, y.b)};
        else if (op == X_MULF)
          r = {mul2(x.v, y.v), add2(mul2(x.a, y.v), mul2(x.v, y.a)), add2(mul2(x.b, y.v), mul2(x.v, y.b))};
        else if (op == X_DIVF) {
          r.v = f2(__fdiv_rn(x.v.x, y.v.x), __fdiv_rn(x.v.y, y.v.y));
          r.a = f2(__fdiv_rn(x.a.x - r.v.x * y.a.x, y.v.x), __fdiv_rn(x.a.y - r.v.y * y.a.y, y.v.y));
          r.b = f2(__fdiv_rn(x.b.x - r.v.x * y.b.x, y.v.x), __fdiv_rn(x.b.y - r.v.y * y.b.y, y.v.y));
        } else {
          const bool mx = op == X_MAXF;
          const float2 c = fl2(int(mx ? y.v.x > x.v.x : y.v.x < x.v.x), int(mx ? y.v.y > x.v.y : y.v.y < x.v.y));
          r = {sel2(c, y.v, x.v), sel2(c, y.a, x.a), sel2(c, y.b, x.b)};
        }
        tos = r;
        ++pc;
        break;
      }
      case X_LTF: case X_LEF: case X_EQF: {
        const TV y = pop(), x = tos;
        const float2 p = op == X_LTF ? fl2(int(x.v.x < y.v.x), int(x.v.y < y.v.y))
                         : op == X_LEF ? fl2(int(x.v.x <= y.v.x), int(x.v.y <= y.v.y))
                                       : fl2(int(x.v.x == y.v.x), int(x.v.y == y.v.y));
        tos = tv(p);
        ++pc;
        break;
      }
      case X_ADDI: case X_SUBI: case X_MULI: case X_MAXI: case X_MINI: case X_LTI: case X_LEI:
      case X_EQI: case X_AND: case X_OR: {
        const TV y = pop(), x = tos;
        int r[2];
        const int xa[2] = {bits(x.v.x), bits(x.v.y)}, ya[2] = {bits(y.v.x), bits(y.v.y)};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int a_ = xa[q], b_ = ya[q];
          r[q] = op == X_ADDI ? a_ + b_ : op == X_SUBI ? (a_ > b_ ? a_ - b_ : 0) : op == X_MULI ? a_ * b_
               : op == X_MAXI ? (a_ > b_ ? a_ : b_) : op == X_MINI ? (a_ < b_ ? a_ : b_)
               : op == X_LTI ? int(a_ < b_) : op == X_LEI ? int(a_ <= b_) : op == X_EQI ? int(a_ == b_)
               : op == X_AND ? (a_ & b_) : (a_ | b_);
        }
        tos = tv(fl2(r[0], r[1]));
        ++pc;
        break;
      }
      case X_ADDFK: case X_SUBFK: case X_MULFK: case X_DIVFK: case X_MAXFK: case X_MINFK:
      case X_RSUBFK: case X_RDIVFK: {
        const TV x = tos;
        TV r;
        if (op == X_ADDFK) r = {f2(x.v.x + kk, x.v.y + kk), x.a, x.b};
        else if (op == X_SUBFK) r = {f2(x.v.x - kk, x.v.y - kk), x.a, x.b};
        else if (op == X_MULFK) r = {scl2(x.v, kk), scl2(x.a, kk), scl2(x.b, kk)};
        else if (op == X_DIVFK)
          r = {f2(__fdiv_rn(x.v.x, kk), __fdiv_rn(x.v.y, kk)), f2(__fdiv_rn(x.a.x, kk), __fdiv_rn(x.a.y, kk)),
               f2(__fdiv_rn(x.b.x, kk), __fdiv_rn(x.b.y, kk))};
        else if (op == X_RSUBFK) r = {f2(kk - x.v.x, kk - x.v.y), neg2(x.a), neg2(x.b)};
        else if (op == X_RDIVFK) {
          r.v = f2(__fdiv_rn(kk, x.v.x), __fdiv_rn(kk, x.v.y));
          const float2 q = f2(-__fdiv_rn(r.v.x, x.v.x), -__fdiv_rn(r.v.y, x.v.y));
          r.a = mul2(q, x.a);
          r.b = mul2(q, x.b);
        } else {
          const bool mx = op == X_MAXFK;  // literal chosen -> zero tangent
          const float2 c = fl2(int(mx ? kk > x.v.x : kk < x.v.x), int(mx ? kk > x.v.y : kk < x.v.y));
          const float2 z = f2(0.f, 0.f);
          r = {sel2(c, f2(kk, kk), x.v), sel2(c, z, x.a), sel2(c, z, x.b)};
        }
        tos = r;
        ++pc;
        break;
      }
      case X_LTFK: case X_LEFK: case X_EQFK: case X_RLTFK: case X_RLEFK: {
        const float2 x = tos.v;
        const float2 p = op == X_LTFK ? fl2(int(x.x < kk), int(x.y < kk))
                         : op == X_LEFK ? fl2(int(x.x <= kk), int(x.y <= kk))
                         : op == X_EQFK ? fl2(int(x.x == kk), int(x.y == kk))
                         : op == X_RLTFK ? fl2(int(kk < x.x), int(kk < x.y))
                                         : fl2(int(kk <= x.x), int(kk <= x.y));
        tos = tv(p);
        ++pc;
        break;
      }
      case X_IF: {
        const bool c0 = bits(tos.v.x) != 0, c1 = bits(tos.v.y) != 0;
        if (__any_sync(kFull, (live0 && c0) || (live1 && c1))) { ++pc; break; }
        push(tv(f2(0.f, 0.f)));
        pc = int(I.z);
        break;
      }
      case X_ELSE: {
        const float2 c = SL(3 * (sp - 1));
        const bool c0 = bits(c.x) != 0, c1 = bits(c.y) != 0;
        if (__any_sync(kFull, (live0 && !c0) || (live1 && !c1))) { ++pc; break; }
        push(tv(f2(0.f, 0.f)));
        pc = int(I.z);
        break;
      }
      case X_SEL: {
        const TV th = ldv(R, sp - 1);
        const float2 c = SL(3 * (sp - 2));
        sp -= 2;
        tos = {sel2(c, th.v, tos.v), sel2(c, th.a, tos.a), sel2(c, th.b, tos.b)};
        ++pc;
        break;
      }
      case X_LOOP: {
        const int F = int(I.x >> 8);
        fset(F, LF_K, fl2(0, 0));
        fset(F, LF_T0, fl2(t0, t0));
        fset(F, LF_DONE, fl2(live0 ? 0 : 1, live1 ? 0 : 1));
        stv(R, F + LF_RES, tv(f2(0.f, 0.f)));
        ++pc;
        break;
      }
      case X_LOOPANY: {
        const int F = int((I.x >> 8) & 0xffu);
        const float lit = pool[I.x >> 16];
        const uint4 Dsc = P[pc + 1];
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
          push(tv(f2(r0, r1)));
          pc = int(I.w);
          break;
        }
        fset(F, LF_T0, fl2(t0, t0));
        fset(F, LF_DONE, fl2(d0, d1));
        stv(R, F + LF_RES, tv(f2(r0, r1)));
        t0 += n;
        pc += 2;
        break;
      }
      case X_LTEST: {
        const int F = int(I.x >> 8);
        const TV c = pop();
        const float2 d = fget(F, LF_DONE);
        const int n0 = bits(c.v.x) != 0 && bits(d.x) == 0, n1 = bits(c.v.y) != 0 && bits(d.y) == 0;
        fset(F, LF_NEWLY, fl2(n0, n1));
        pc = __any_sync(kFull, n0 | n1) ? pc + 1 : int(I.z);
        break;
      }
      case X_LLATCH: {
        const int F = int(I.x >> 8);
        const TV v = pop();
        const float2 nw = fget(F, LF_NEWLY);
        if (bits(nw.x) | bits(nw.y)) {
          const TV r = ldv(R, F + LF_RES);
          const float2 d = fget(F, LF_DONE);
          stv(R, F + LF_RES, {sel2(nw, v.v, r.v), sel2(nw, v.a, r.a), sel2(nw, v.b, r.b)});
          fset(F, LF_DONE, fl2(bits(d.x) | bits(nw.x), bits(d.y) | bits(nw.y)));
        }
        ++pc;
        break;
      }
      case X_LSTEPK:
      case X_LNEXT: {
        const bool step = op == X_LSTEPK;
        const int F = step ? int((I.x >> 8) & 0xffu) : int(I.x >> 8);
        float2 d = fget(F, LF_DONE);
        if (step) {
          const TV c = pop();
          const int n0 = bits(c.v.x) != 0 && bits(d.x) == 0, n1 = bits(c.v.y) != 0 && bits(d.y) == 0;
          if (n0 | n1) {
            const float lit = pool[I.x >> 16];
            const TV r = ldv(R, F + LF_RES);
            const float2 nw = fl2(n0, n1), z = f2(0.f, 0.f);
            stv(R, F + LF_RES, {sel2(nw, f2(lit, lit), r.v), sel2(nw, z, r.a), sel2(nw, z, r.b)});
            d = fl2(bits(d.x) | n0, bits(d.y) | n1);
            fset(F, LF_DONE, d);
          }
        }
        const int t0e = bits(fget(F, LF_T0).x);
        if (__all_sync(kFull, (bits(d.x) & bits(d.y)) != 0)) {
          t0 = t0e;
          push(ldv(R, F + LF_RES));
          pc = int(I.w);
          break;
        }
        int k = bits(fget(F, LF_K).x);
        if (k == int(I.y)) {
          t0 = t0e + k;
          ++pc;
          break;
        }
        ++k;
        fset(F, LF_K, fl2(k, k));
        t0 = t0e + k;
        pc = int(I.z);
        break;
      }
      case X_LEND: {
        const int F = int(I.x >> 8);
        const float2 d = fget(F, LF_DONE);
        const TV r = ldv(R, F + LF_RES);
        tos = {sel2(d, r.v, tos.v), sel2(d, r.a, tos.a), sel2(d, r.b, tos.b)};
        t0 = bits(fget(F, LF_T0).x);
        ++pc;
        break;
      }
      default:
        return tos;
    }
  }
}

// One launch per underlying g = a.greek_label: per path (x, dx/dS0_g,
// dx/dsigma_g); per tile the FP64 sums and sums of squares of the three, in
// the pricing kernel's deterministic chunked reduction (width 6).
template <int D, bool WRITE>
__global__ void __launch_bounds__(kBlock) greeks_kernel(const PriceArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int last_block;
  uint4 *P = reinterpret_cast<uint4 *>(smem);
  const int prog_words = a.n_insn * 4 + a.n_pool;
  const uint32_t *src = reinterpret_cast<const uint32_t *>(a.prog);
  for (int i = threadIdx.x; i < prog_words; i += blockDim.x) smem[i] = src[i];
  __syncthreads();
  const float *pool = reinterpret_cast<const float *>(smem + a.n_insn * 4);
  float2 *R = reinterpret_cast<float2 *>(smem + prog_words) + threadIdx.x;
  float Bm[D * D], S0[D], Lm[D * D];
  load_model_regs<D>(a.m, Bm, S0);
#pragma unroll
  for (int i = 0; i < D * D; ++i) Lm[i] = __ldg(a.m.L + i);
  const int gl = a.greek_label;
  const float sig_g = __ldg(a.m.sig + gl);
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
    const TV x = eval_greeks<D>(P, pool, R, a, g, live0, live1, Bm, S0, Lm, gl, sig_g);
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

template <typename K>
cudaError_t set_smem_g(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

}  // namespace

cudaError_t launch_greeks(const PriceArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
  const bool w = a.out_paths != nullptr;
#define GLAUNCH(DD, WW)                                                            \
  do {                                                                             \
    auto k = greeks_kernel<DD, WW>;                                                \
    cudaError_t e = set_smem_g(k, smem);                                           \
    if (e != cudaSuccess) return e;                                                \
    k<<<grid, block, smem, s>>>(a);                                                \
    return cudaGetLastError();                                                     \
  } while (0)
  switch (a.m.d) {
    case 1: if (w) GLAUNCH(1, true); else GLAUNCH(1, false);
    case 2: if (w) GLAUNCH(2, true); else GLAUNCH(2, false);
    case 3: if (w) GLAUNCH(3, true); else GLAUNCH(3, false);
    case 4: if (w) GLAUNCH(4, true); else GLAUNCH(4, false);
    default: return cudaErrorInvalidValue;
  }
#undef GLAUNCH
}

int greeks_blocks_per_sm(int d, int block, size_t smem) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define GOCC(DD)                                                                             \
  set_smem_g(greeks_kernel<DD, false>, smem);                                                \
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, greeks_kernel<DD, false>, block, smem)
  switch (d) {
    case 1: GOCC(1); break;
    case 2: GOCC(2); break;
    case 3: GOCC(3); break;
    case 4: GOCC(4); break;
    default: return 0;
  }
#undef GOCC
  return e == cudaSuccess ? nb : 0;
}

}  // namespace pc
