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
  const ModelDev &m = a.m;
  const Layout &lay = a.lay;
  PathState<D> ps;
  path_state_init<D>(ps, R, lay);
  const int t_now = m.t_now;
  int pc = 0, sp = 0, t0 = 0;
  float2 tos = make_float2(0.f, 0.f);
  int tid = -1;  // entry of tos
  // logical slot s: value at physical slot 2s, entry number at 2s + 1
  auto sv = [&](int s) -> float2 & { return SL(2 * s); };
  auto sid_get = [&](int s) { return __float_as_int(SL(2 * s + 1).x); };
  auto sid_set = [&](int s, int e) { SL(2 * s + 1) = make_float2(__int_as_float(e), 0.f); };
  auto push = [&](float2 v, int e) {
    sv(sp) = tos;
    sid_set(sp, tid);
    ++sp;
    tos = v;
    tid = e;
  };
  auto pop = [&](int &e) {
    const float2 v = tos;
    e = tid;
    --sp;
    tos = sv(sp);
    tid = sid_get(sp);
    return v;
  };
  auto ensure = [&](int &o) {
    if (o > m.n || o < -m.n_hist) {
      atomicOr(a.status, 1);
      o = o > m.n ? m.n : -m.n_hist;
    }
    while (ps.f < o) gen_date<D, true>(ps.f + 1, ps, m, lay, g, R, Bm, S0, Lm);
  };
  auto read = [&](int o, int l) -> float2 {
    if (o > 0) return SL(lay.off_win + (o & (lay.win - 1)) * D + l);
    const float v = __ldg(m.sval + (o + m.n_hist) * D + l);
    return make_float2(v, v);
  };
  const float2 one = make_float2(1.f, 1.f), zero = make_float2(0.f, 0.f);
  for (;;) {
    const uint4 I = P[pc];
    const uint32_t op = I.x & 0xffu;
    const float kk = __uint_as_float(I.y);
    switch (op) {
      case X_CONST: push(make_float2(kk, kk), -1); ++pc; break;
      case X_MODEL:
      case X_MODEL_MULK:
      case X_MODEL_DIVK: {
        int o = int(I.y) + t0 - t_now;
        ensure(o);
        int l = int(I.x >> 8) & 3;
        l = l < D ? l : 0;
        float2 v = read(o, l);
        const float k = __uint_as_float(I.z);
        const float2 s = v;
        float scale = 1.f;
        if (op == X_MODEL_MULK) {
          v = make_float2(__fmul_rn(v.x, k), __fmul_rn(v.y, k));
          scale = k;
        } else if (op == X_MODEL_DIVK) {
          v = make_float2(__fdiv_rn(v.x, k), __fdiv_rn(v.y, k));
          scale = __frcp_rn(k);
        }
        push(v, adj_leaf<D>(T, o, l, s, scale, R, m, lay, S0));
        ++pc;
        break;
      }
      case X_LRED:
      case X_LANY: {
        int o = int(I.y) + t0 - t_now;
        ensure(o);
        const uint32_t A = I.x >> 8;
        const int code = int((A >> 4) & 7u);
        if (op == X_LANY || code) {  // a test: boolean, no derivative
          push(fused_value<D>(I, o, pool, R, m, lay), -1);
          ++pc;
          break;
        }
        const int n = int((A >> 8) & 3u) + 1, kind = int((A >> 2) & 3u), rop = int(A & 3u);
        float2 v = zero;
        int e = -1;
        for (int i = 0; i < n; ++i) {
          int l = int(A >> (10 + 2 * i)) & 3;
          l = l < D ? l : 0;
          const float2 s0 = read(o, l);
          float2 s = s0;
          float scale = 1.f;
          if (kind == 1) {
            const float c = pool[I.z + i];
            s = make_float2(__fmul_rn(s.x, c), __fmul_rn(s.y, c));
            scale = c;
          } else if (kind == 2) {
            const float c = pool[I.z + i];
            s = make_float2(__fdiv_rn(s.x, c), __fdiv_rn(s.y, c));
            scale = __frcp_rn(c);
          }
          const int el = adj_leaf<D>(T, o, l, s0, scale, R, m, lay, S0);
          if (i == 0) {
            v = s;
            e = el;
          } else if (rop == 2) {
            v = make_float2(__fadd_rn(v.x, s.x), __fadd_rn(v.y, s.y));
            e = T.add(e, el, one, one);
          } else {
            // the leaf taken when it is strictly beyond the running value
            const float2 t = fl2(int(rop == 0 ? s.x < v.x : s.x > v.x), int(rop == 0 ? s.y < v.y : s.y > v.y));
            v = rop == 0 ? make_float2(fminf(v.x, s.x), fminf(v.y, s.y)) : make_float2(fmaxf(v.x, s.x), fmaxf(v.y, s.y));
            e = T.add(e, el, adsel(t, zero, one), adsel(t, one, zero));
          }
        }
        push(v, e);
        ++pc;
        break;
      }
      case X_PAYOFF: {
        int o = int(I.y) + t0 - t_now;
        if (o > m.n || o < -m.n_hist) {
          atomicOr(a.status, 1);
          o = 0;
        }
        float v = __fmul_rn(__uint_as_float(I.z), __ldg(m.disc + o + m.n_hist));
        if (I.x >> 8) v = -v;
        push(make_float2(v, v), -1);
        ++pc;
        break;
      }
      case X_TIME: push(fl2(int(I.y) + t0, int(I.y) + t0), -1); ++pc; break;
      case X_NOW: push(fl2(t_now, t_now), -1); ++pc; break;
      case X_NEGF:
        tos = make_float2(-tos.x, -tos.y);
        tid = T.add(tid, -1, make_float2(-1.f, -1.f), zero);
        ++pc;
        break;
      case X_NOT: tos = fl2(bits(tos.x) ^ 1, bits(tos.y) ^ 1); ++pc; break;
      case X_ADDF: case X_SUBF: case X_MULF: case X_DIVF: case X_MAXF: case X_MINF: {
        int ey;
        const float2 y = pop(ey), x = tos;
        const int ex = tid;
        float2 r, p1, p2;
        if (op == X_ADDF) {
          r = make_float2(__fadd_rn(x.x, y.x), __fadd_rn(x.y, y.y));
          p1 = one;
          p2 = one;
        } else if (op == X_SUBF) {
          r = make_float2(__fsub_rn(x.x, y.x), __fsub_rn(x.y, y.y));
          p1 = one;
          p2 = make_float2(-1.f, -1.f);
        } else if (op == X_MULF) {
          r = make_float2(__fmul_rn(x.x, y.x), __fmul_rn(x.y, y.y));
          p1 = y;
          p2 = x;
        } else if (op == X_DIVF) {
          r = make_float2(__fdiv_rn(x.x, y.x), __fdiv_rn(x.y, y.y));
          p1 = make_float2(__frcp_rn(y.x), __frcp_rn(y.y));
          p2 = make_float2(-__fdiv_rn(r.x, y.x), -__fdiv_rn(r.y, y.y));
        } else {
          const bool mx = op == X_MAXF;
          const float2 t = fl2(int(mx ? y.x > x.x : y.x < x.x), int(mx ? y.y > x.y : y.y < x.y));
          r = mx ? make_float2(fmaxf(x.x, y.x), fmaxf(x.y, y.y)) : make_float2(fminf(x.x, y.x), fminf(x.y, y.y));
          p1 = adsel(t, zero, one);
          p2 = adsel(t, one, zero);
        }
        tos = r;
        tid = T.add(ex, ey, p1, p2);
        ++pc;
        break;
      }
      case X_LTF: case X_LEF: case X_EQF: {
        int ey;
        const float2 y = pop(ey), x = tos;
        tos = op == X_LTF ? fl2(int(x.x < y.x), int(x.y < y.y))
              : op == X_LEF ? fl2(int(x.x <= y.x), int(x.y <= y.y))
                            : fl2(int(x.x == y.x), int(x.y == y.y));
        tid = -1;
        ++pc;
        break;
      }
      case X_ADDI: case X_SUBI: case X_MULI: case X_MAXI: case X_MINI: case X_LTI: case X_LEI:
      case X_EQI: case X_AND: case X_OR: {
        int ey;
        const float2 y = pop(ey), x = tos;
        int r[2];
        const int xa[2] = {bits(x.x), bits(x.y)}, ya[2] = {bits(y.x), bits(y.y)};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int a_ = xa[q], b_ = ya[q];
          r[q] = op == X_ADDI ? a_ + b_ : op == X_SUBI ? (a_ > b_ ? a_ - b_ : 0) : op == X_MULI ? a_ * b_
               : op == X_MAXI ? (a_ > b_ ? a_ : b_) : op == X_MINI ? (a_ < b_ ? a_ : b_)
               : op == X_LTI ? int(a_ < b_) : op == X_LEI ? int(a_ <= b_) : op == X_EQI ? int(a_ == b_)
               : op == X_AND ? (a_ & b_) : (a_ | b_);
        }
        tos = fl2(r[0], r[1]);
        tid = -1;
        ++pc;
        break;
      }
      case X_ADDFK: case X_SUBFK: case X_MULFK: case X_DIVFK: case X_MAXFK: case X_MINFK:
      case X_RSUBFK: case X_RDIVFK: {
        const float2 x = tos;
        float2 r, p;
        if (op == X_ADDFK) {
          r = make_float2(__fadd_rn(x.x, kk), __fadd_rn(x.y, kk));
          p = one;
        } else if (op == X_SUBFK) {
          r = make_float2(__fsub_rn(x.x, kk), __fsub_rn(x.y, kk));
          p = one;
        } else if (op == X_MULFK) {
          r = make_float2(__fmul_rn(x.x, kk), __fmul_rn(x.y, kk));
          p = make_float2(kk, kk);
        } else if (op == X_DIVFK) {
          r = make_float2(__fdiv_rn(x.x, kk), __fdiv_rn(x.y, kk));
          const float q = __frcp_rn(kk);
          p = make_float2(q, q);
        } else if (op == X_RSUBFK) {
          r = make_float2(__fsub_rn(kk, x.x), __fsub_rn(kk, x.y));
          p = make_float2(-1.f, -1.f);
        } else if (op == X_RDIVFK) {
          r = make_float2(__fdiv_rn(kk, x.x), __fdiv_rn(kk, x.y));
          p = make_float2(-__fdiv_rn(r.x, x.x), -__fdiv_rn(r.y, x.y));
        } else {  // the literal taken: no derivative
          const bool mx = op == X_MAXFK;
          const float2 t = fl2(int(mx ? kk > x.x : kk < x.x), int(mx ? kk > x.y : kk < x.y));
          r = mx ? make_float2(fmaxf(x.x, kk), fmaxf(x.y, kk)) : make_float2(fminf(x.x, kk), fminf(x.y, kk));
          p = adsel(t, zero, one);
        }
        tos = r;
        tid = T.add(tid, -1, p, zero);
        ++pc;
        break;
      }
      case X_LTFK: case X_LEFK: case X_EQFK: case X_RLTFK: case X_RLEFK: {
        const float2 x = tos;
        tos = op == X_LTFK ? fl2(int(x.x < kk), int(x.y < kk))
              : op == X_LEFK ? fl2(int(x.x <= kk), int(x.y <= kk))
              : op == X_EQFK ? fl2(int(x.x == kk), int(x.y == kk))
              : op == X_RLTFK ? fl2(int(kk < x.x), int(kk < x.y))
                              : fl2(int(kk <= x.x), int(kk <= x.y));
        tid = -1;
        ++pc;
        break;
      }
      case X_IF: {
        const bool c0 = bits(tos.x) != 0, c1 = bits(tos.y) != 0;
        if (__any_sync(kFull, (live0 && c0) || (live1 && c1))) { ++pc; break; }
        push(zero, -1);
        pc = int(I.z);
        break;
      }
      case X_ELSE: {
        const float2 c = sv(sp - 1);
        const bool c0 = bits(c.x) != 0, c1 = bits(c.y) != 0;
        if (__any_sync(kFull, (live0 && !c0) || (live1 && !c1))) { ++pc; break; }
        push(zero, -1);
        pc = int(I.z);
        break;
      }
      case X_SEL: {
        const float2 th = sv(sp - 1), c = sv(sp - 2);
        const int eth = sid_get(sp - 1);
        sp -= 2;
        const float2 ct = fl2(bits(c.x) != 0, bits(c.y) != 0);
        tid = T.add(eth, tid, adsel(ct, one, zero), adsel(ct, zero, one));
        tos = adsel(ct, th, tos);
        ++pc;
        break;
      }
      case X_LOOP: {
        const int F = int(I.x >> 8);
        sv(F + LF_K) = fl2(0, 0);
        sv(F + LF_T0) = fl2(t0, t0);
        sv(F + LF_DONE) = fl2(live0 ? 0 : 1, live1 ? 0 : 1);
        sv(F + LF_RES) = zero;
        sid_set(F + LF_RES, -1);
        ++pc;
        break;
      }
      case X_LOOPANY: {
        const int F = int((I.x >> 8) & 0xffu);
        const float lit = pool[I.x >> 16];
        const uint4 Dsc = P[pc + 1];
        bool d0 = !live0, d1 = !live1;
        float r0 = 0.f, r1 = 0.f;
        int n = int(I.y);
        bool all = false;
        int o0 = int(Dsc.y) + t0 - t_now;
        if (o0 < -m.n_hist || o0 + n > m.n) {
          atomicOr(a.status, 1);
          o0 = o0 < -m.n_hist ? -m.n_hist : o0 > m.n ? m.n : o0;
          n = o0 + n > m.n ? m.n - o0 : n;
        }
        for (int k = 0;; ++k) {
          const int o = o0 + k;
          while (ps.f < o) gen_date<D, true>(ps.f + 1, ps, m, lay, g, R, Bm, S0, Lm);
          const float2 c = fused_value<D>(Dsc, o, pool, R, m, lay);
          if (bits(c.x) && !d0) { d0 = true; r0 = lit; }
          if (bits(c.y) && !d1) { d1 = true; r1 = lit; }
          all = __all_sync(kFull, d0 && d1);
          if (all || k == n) break;
        }
        if (all) {
          push(make_float2(r0, r1), -1);
          pc = int(I.w);
          break;
        }
        sv(F + LF_T0) = fl2(t0, t0);
        sv(F + LF_DONE) = fl2(d0, d1);
        sv(F + LF_RES) = make_float2(r0, r1);
        sid_set(F + LF_RES, -1);
        t0 += n;
        pc += 2;
        break;
      }
      case X_LTEST: {
        const int F = int(I.x >> 8);
        int ec;
        const float2 c = pop(ec);
        const float2 d = sv(F + LF_DONE);
        const int n0 = bits(c.x) != 0 && bits(d.x) == 0, n1 = bits(c.y) != 0 && bits(d.y) == 0;
        sv(F + LF_NEWLY) = fl2(n0, n1);
        pc = __any_sync(kFull, n0 | n1) ? pc + 1 : int(I.z);
        break;
      }
      case X_LLATCH: {
        const int F = int(I.x >> 8);
        int ev;
        const float2 v = pop(ev);
        const float2 nw = sv(F + LF_NEWLY);
        if (__any_sync(kFull, (bits(nw.x) | bits(nw.y)) != 0)) {  // uniform: an entry for the warp
          const float2 r = sv(F + LF_RES), d = sv(F + LF_DONE);
          const float2 nt = fl2(bits(nw.x) != 0, bits(nw.y) != 0);
          const int er = T.add(ev, sid_get(F + LF_RES), adsel(nt, one, zero), adsel(nt, zero, one));
          sv(F + LF_RES) = adsel(nt, v, r);
          sid_set(F + LF_RES, er);
          sv(F + LF_DONE) = fl2(bits(d.x) | bits(nw.x), bits(d.y) | bits(nw.y));
        }
        ++pc;
        break;
      }
      case X_LSTEPK:
      case X_LNEXT: {
        const bool step = op == X_LSTEPK;
        const int F = step ? int((I.x >> 8) & 0xffu) : int(I.x >> 8);
        float2 d = sv(F + LF_DONE);
        if (step) {  // latch the literal (no derivative) on newly true lanes
          int ec;
          const float2 c = pop(ec);
          const int n0 = bits(c.x) != 0 && bits(d.x) == 0, n1 = bits(c.y) != 0 && bits(d.y) == 0;
          if (__any_sync(kFull, (n0 | n1) != 0)) {
            const float lit = pool[I.x >> 16];
            const float2 r = sv(F + LF_RES), nt = fl2(n0, n1);
            const int er = T.add(-1, sid_get(F + LF_RES), zero, adsel(nt, zero, one));
            sv(F + LF_RES) = adsel(nt, make_float2(lit, lit), r);
            sid_set(F + LF_RES, er);
            d = fl2(bits(d.x) | n0, bits(d.y) | n1);
            sv(F + LF_DONE) = d;
          }
        }
        const int t0e = bits(sv(F + LF_T0).x);
        if (__all_sync(kFull, (bits(d.x) & bits(d.y)) != 0)) {
          t0 = t0e;
          push(sv(F + LF_RES), sid_get(F + LF_RES));
          pc = int(I.w);
          break;
        }
        int k = bits(sv(F + LF_K).x);
        if (k == int(I.y)) {
          t0 = t0e + k;
          ++pc;
          break;
        }
        ++k;
        sv(F + LF_K) = fl2(k, k);
        t0 = t0e + k;
        pc = int(I.z);
        break;
      }
      case X_LEND: {
        const int F = int(I.x >> 8);
        const float2 d = sv(F + LF_DONE), r = sv(F + LF_RES);
        const float2 dt = fl2(bits(d.x) != 0, bits(d.y) != 0);
        tid = T.add(sid_get(F + LF_RES), tid, adsel(dt, one, zero), adsel(dt, zero, one));
        tos = adsel(dt, r, tos);
        t0 = bits(sv(F + LF_T0).x);
        ++pc;
        break;
      }
      default:
        res = tid;
        return tos;
    }
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
template <int D, bool WRITE>
__device__ __forceinline__ void adjoint_tiles(const PriceArgs &a, const TapeArgs &ta) {
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
    const float2 x = eval_adjoint<D>(P, pool, R, a, g, live0, live1, Bm, S0, Lm, T, res);
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
