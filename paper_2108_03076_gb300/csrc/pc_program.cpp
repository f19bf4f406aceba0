// pc_program.cpp -- payoff programs on the host: text assembler, bytecode
// decoder / verifier / binder, emission of the executable form run by the
// kernel, and the static time analysis against a model.
//
// The language is the payoff intermediate language of Sec. 3 with the
// semantics of Fig. 3; values are nats, reals and bools; template variables
// (Sec. 2) are bound at load time so every time expression becomes a static
// integer; payoff(t, p1', p2') is folded to +d(t), -d(t) or 0 for the
// two-party view (p1, p2) of Fig. 3.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>

#include "pc_internal.h"

namespace pc {

namespace {

enum Ty : uint8_t { T_REAL = 1, T_BOOL = 2, T_NAT = 3 };

struct TNode {
  uint32_t op = 0;        // pc_opcode
  Ty ty = T_REAL;
  int32_t a = 0;          // label / bool / nat value
  int64_t time = 0;       // bound static time (T[t]delta)
  int32_t sign = 0;       // payoff sign after party folding
  double val = 0;         // real literal
  int32_t ch[3] = {-1, -1, -1};
  int32_t nch = 0;
};

uint32_t fbits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

struct Decoder {
  const uint32_t *w;
  size_t n, i = 0;
  const int32_t *tp;
  size_t ntp;
  int32_t max_tp = 0;
  std::string &err;

  Decoder(const uint32_t *w_, size_t n_, const int32_t *tp_, size_t ntp_, std::string &e)
      : w(w_), n(n_), tp(tp_), ntp(ntp_), err(e) {}

  // TIME operand: count word then terms.  kind 0: ILTExprZ (any integer),
  // 1: ILTExpr (natural), 2: TExpr (one literal or one variable).
  pc_status time(int kind, int64_t &out) {
    if (i >= n) { err = "truncated time expression"; return PC_EBYTECODE; }
    uint32_t c = w[i++];
    if (c == 0 || c > 16) { err = "time expression needs 1..16 terms"; return PC_EBYTECODE; }
    if (kind == 2 && c != 1) { err = "loopif bound must be one literal or one variable"; return PC_EBYTECODE; }
    if (i + c > n) { err = "truncated time expression"; return PC_EBYTECODE; }
    int64_t s = 0;
    for (uint32_t k = 0; k < c; ++k) {
      uint32_t t = w[i++];
      if (t & 0x80000000u) {
        uint32_t v = t & 0x7fffffffu;
        if (v >= ntp) { err = "template variable $" + std::to_string(v) + " is not bound"; return PC_ETPARAM; }
        if (tp[v] < 0) { err = "template variable $" + std::to_string(v) + " is negative"; return PC_ETPARAM; }
        max_tp = std::max<int32_t>(max_tp, int32_t(v) + 1);
        s += tp[v];
      } else {
        int32_t lit = int32_t(t << 1) >> 1;  // sign-extend 31 bits
        if (kind != 0 && lit < 0) { err = "negative literal in a natural time expression"; return PC_EBYTECODE; }
        s += lit;
      }
    }
    if (s < -(int64_t(1) << 30) || s > (int64_t(1) << 30)) { err = "time expression out of range"; return PC_ERANGE; }
    out = s;
    return PC_OK;
  }
};

bool is_arith(uint32_t op) { return op == PC_OP_ADD || op == PC_OP_SUB || op == PC_OP_MULT; }

pc_status typecheck(std::vector<TNode> &T, int root, std::string &err) {
  // children precede parents in postfix order, so a forward pass suffices
  for (size_t k = 0; k < T.size(); ++k) {
    TNode &x = T[k];
    auto ty = [&](int c) { return T[x.ch[c]].ty; };
    switch (x.op) {
      case PC_OP_REAL: x.ty = T_REAL; break;
      case PC_OP_BOOL: x.ty = T_BOOL; break;
      case PC_OP_NAT: case PC_OP_NOW: case PC_OP_TEXPR: x.ty = T_NAT; break;
      case PC_OP_MODEL: case PC_OP_PAYOFF: x.ty = T_REAL; break;
      case PC_OP_NEG:
        if (ty(0) != T_REAL) { err = "neg needs a real"; return PC_EBYTECODE; }
        x.ty = T_REAL; break;
      case PC_OP_NOT:
        if (ty(0) != T_BOOL) { err = "not needs a bool"; return PC_EBYTECODE; }
        x.ty = T_BOOL; break;
      case PC_OP_ADD: case PC_OP_SUB: case PC_OP_MULT: case PC_OP_MAX: case PC_OP_MIN:
        if (ty(0) != ty(1) || ty(0) == T_BOOL) { err = "arithmetic needs two reals or two nats"; return PC_EBYTECODE; }
        x.ty = ty(0); break;
      case PC_OP_DIV:
        if (ty(0) != T_REAL || ty(1) != T_REAL) { err = "div needs two reals"; return PC_EBYTECODE; }
        x.ty = T_REAL; break;
      case PC_OP_LT: case PC_OP_LE:
        if (ty(0) != ty(1) || ty(0) == T_BOOL) { err = "comparison needs two reals or two nats"; return PC_EBYTECODE; }
        x.ty = T_BOOL; break;
      case PC_OP_EQ:
        if (ty(0) != ty(1)) { err = "eq needs operands of one type"; return PC_EBYTECODE; }
        x.ty = T_BOOL; break;
      case PC_OP_AND: case PC_OP_OR:
        if (ty(0) != T_BOOL || ty(1) != T_BOOL) { err = "and/or need bools"; return PC_EBYTECODE; }
        x.ty = T_BOOL; break;
      case PC_OP_IF: case PC_OP_LOOPIF:
        if (ty(0) != T_BOOL) { err = "if/loopif condition must be a bool"; return PC_EBYTECODE; }
        if (ty(1) != ty(2)) { err = "if/loopif branches have different types"; return PC_EBYTECODE; }
        x.ty = ty(1); break;
      default: err = "internal: unknown node"; return PC_EBYTECODE;
    }
  }
  if (T[root].ty != T_REAL) { err = "a payoff expression must be real-valued"; return PC_EBYTECODE; }
  return PC_OK;
}

struct Emitter {
  const std::vector<TNode> &T;
  std::vector<XInsn> code;
  std::vector<float> pool;
  int depth = 0, max_depth = 0, nest = 0, max_nest = 0, n_loops = 0;

  explicit Emitter(const std::vector<TNode> &t) : T(t) {}

  // --- fused multi-asset ops ------------------------------------------------
  // An S-term is model(l, t), model(l, t) * k, k * model(l, t) or
  // model(l, t) / k with k a real literal.
  struct STerm {
    int label;
    int64_t time;
    int kind;  // 0 none, 1 mult, 2 div
    float k;
  };
  bool sterm(int idx, STerm &s) const {
    const TNode &x = T[idx];
    if (x.op == PC_OP_MODEL) { s = {x.a, x.time, 0, 1.f}; return true; }
    if ((x.op == PC_OP_MULT || x.op == PC_OP_DIV) && x.ty == T_REAL) {
      const TNode &a = T[x.ch[0]], &b = T[x.ch[1]];
      const int kind = x.op == PC_OP_MULT ? 1 : 2;
      // a scale of exactly 1 is no scale (x * 1 and x / 1 are exact)
      if (a.op == PC_OP_MODEL && b.op == PC_OP_REAL) {
        s = {a.a, a.time, float(b.val) == 1.0f ? 0 : kind, float(b.val)};
        return true;
      }
      if (kind == 1 && b.op == PC_OP_MODEL && a.op == PC_OP_REAL) {
        s = {b.a, b.time, float(a.val) == 1.0f ? 0 : 1, float(a.val)};
        return true;
      }
    }
    return false;
  }
  // Leaves of the left-nested chain of `op` rooted at idx, in evaluation order.
  void chain(int idx, uint32_t op, std::vector<int> &leaves) const {
    std::vector<int> rights;
    int y = idx;
    while (T[y].op == op && T[y].ty == T[idx].ty) {
      rights.push_back(T[y].ch[1]);
      y = T[y].ch[0];
    }
    leaves.assign(1, y);
    for (auto it = rights.rbegin(); it != rights.rend(); ++it) leaves.push_back(*it);
  }
  // S-terms of one time with compatible scales; returns the common kind or -1.
  int terms_kind(const std::vector<STerm> &ts) const {
    bool mult = false, div = false;
    for (const STerm &t : ts) {
      if (t.time != ts[0].time || t.label < 0 || t.label > 3) return -1;
      mult |= t.kind == 1;
      div |= t.kind == 2;
    }
    if (mult && div) return -1;
    return mult ? 1 : div ? 2 : 0;
  }
  uint32_t pool_terms(const std::vector<STerm> &ts, int kind) {
    const uint32_t off = uint32_t(pool.size());
    if (kind) for (const STerm &t : ts) pool.push_back(t.kind ? t.k : 1.0f);
    return off;
  }
  static uint32_t labels_field(const std::vector<STerm> &ts) {
    uint32_t f = 0;
    for (size_t i = 0; i < ts.size(); ++i) f |= uint32_t(ts[i].label) << (10 + 2 * i);
    return f;
  }
  // chain of min/max/add over S-terms (1..4 leaves; 1 leaf only with a compare)
  bool red_terms(int idx, uint32_t &rop, std::vector<STerm> &ts) const {
    const TNode &x = T[idx];
    ts.clear();
    STerm s;
    if (sterm(idx, s)) { rop = 0; ts.push_back(s); return true; }
    if (x.ty != T_REAL || !(x.op == PC_OP_MIN || x.op == PC_OP_MAX || x.op == PC_OP_ADD)) return false;
    std::vector<int> leaves;
    chain(idx, x.op, leaves);
    if (leaves.size() < 2 || leaves.size() > 4) return false;
    for (int l : leaves) {
      if (!sterm(l, s)) return false;
      ts.push_back(s);
    }
    rop = x.op == PC_OP_MIN ? 0 : x.op == PC_OP_MAX ? 1 : 2;
    return true;
  }
  // compare of an operand with a real literal: code 1 v<k, 2 v<=k, 3 k<v, 4 k<=v
  bool lit_cmp(int idx, int &operand, int &code, float &k) const {
    const TNode &x = T[idx];
    if (!(x.op == PC_OP_LT || x.op == PC_OP_LE)) return false;
    const TNode &a = T[x.ch[0]], &b = T[x.ch[1]];
    if (a.ty != T_REAL) return false;
    if (b.op == PC_OP_REAL && a.op != PC_OP_REAL) {
      operand = x.ch[0]; code = x.op == PC_OP_LT ? 1 : 2; k = float(b.val); return true;
    }
    if (a.op == PC_OP_REAL && b.op != PC_OP_REAL) {
      operand = x.ch[1]; code = x.op == PC_OP_LT ? 3 : 4; k = float(a.val); return true;
    }
    return false;
  }
  static uint32_t fbits_(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }
  bool try_fused(int idx) {
    const TNode &x = T[idx];
    uint32_t rop;
    std::vector<STerm> ts;
    // label reduce without compare
    if (x.ty == T_REAL && (x.op == PC_OP_MIN || x.op == PC_OP_MAX || x.op == PC_OP_ADD) &&
        red_terms(idx, rop, ts) && ts.size() >= 2) {
      const int kind = terms_kind(ts);
      if (kind < 0) return false;
      const uint32_t off = pool_terms(ts, kind);
      emit(X_LRED, rop | (uint32_t(kind) << 2) | (uint32_t(ts.size() - 1) << 8) | labels_field(ts),
           uint32_t(int32_t(ts[0].time)), off, 0);
      push();
      return true;
    }
    // (label reduce or single S-term) compared with a literal
    int operand, code;
    float k;
    if (lit_cmp(idx, operand, code, k) && red_terms(operand, rop, ts)) {
      const int kind = terms_kind(ts);
      if (kind < 0) return false;
      const uint32_t off = pool_terms(ts, kind);
      emit(X_LRED, rop | (uint32_t(kind) << 2) | (uint32_t(code) << 4) |
                       (uint32_t(ts.size() - 1) << 8) | labels_field(ts),
           uint32_t(int32_t(ts[0].time)), off, fbits_(k));
      push();
      return true;
    }
    // or / and of S-term compares against one literal
    if (x.ty == T_BOOL && (x.op == PC_OP_OR || x.op == PC_OP_AND)) {
      std::vector<int> leaves;
      chain(idx, x.op, leaves);
      if (leaves.size() < 2 || leaves.size() > 4) return false;
      int code0 = -1;
      float k0 = 0.f;
      for (int l : leaves) {
        int opd, c;
        float kk;
        STerm st;
        if (!lit_cmp(l, opd, c, kk) || !sterm(opd, st)) return false;
        if (code0 < 0) { code0 = c; k0 = kk; }
        if (c != code0 || fbits_(kk) != fbits_(k0)) return false;
        ts.push_back(st);
      }
      const int kind = terms_kind(ts);
      if (kind < 0) return false;
      const uint32_t off = pool_terms(ts, kind);
      emit(X_LANY, (x.op == PC_OP_AND ? 1u : 0u) | (uint32_t(kind) << 2) | (uint32_t(code0) << 4) |
                       (uint32_t(ts.size() - 1) << 8) | labels_field(ts),
           uint32_t(int32_t(ts[0].time)), off, fbits_(k0));
      push();
      return true;
    }
    return false;
  }

  size_t emit(uint32_t op, uint32_t A = 0, uint32_t b = 0, uint32_t c = 0, uint32_t e = 0) {
    code.push_back({op | (A << 8), b, c, e});
    return code.size() - 1;
  }
  void push() { max_depth = std::max(max_depth, ++depth); }
  void pop(int k = 1) { depth -= k; }

  static bool real_lit(const TNode &x) { return x.op == PC_OP_REAL; }

  void node(int k) {
    const TNode &x = T[k];
    switch (x.op) {
      case PC_OP_REAL: emit(X_CONST, 0, fbits(float(x.val))); push(); return;
      case PC_OP_BOOL: case PC_OP_NAT: emit(X_CONST, 0, uint32_t(x.a)); push(); return;
      case PC_OP_NOW: emit(X_NOW); push(); return;
      case PC_OP_TEXPR: emit(X_TIME, 0, uint32_t(int32_t(x.time))); push(); return;
      case PC_OP_MODEL: emit(X_MODEL, uint32_t(x.a), uint32_t(int32_t(x.time))); push(); return;
      case PC_OP_PAYOFF:
        if (x.sign == 0) emit(X_CONST, 0, fbits(0.f));
        else emit(X_PAYOFF, x.sign < 0 ? 1u : 0u, uint32_t(int32_t(x.time)), fbits(1.0f));
        push();
        return;
      case PC_OP_NEG: node(x.ch[0]); emit(X_NEGF); return;
      case PC_OP_NOT: node(x.ch[0]); emit(X_NOT); return;
      case PC_OP_IF: {
        node(x.ch[0]);
        size_t i_if = emit(X_IF);
        node(x.ch[1]);
        size_t i_else = emit(X_ELSE);
        node(x.ch[2]);
        size_t i_sel = emit(X_SEL);
        code[i_if].c = uint32_t(i_else + 1);
        code[i_else].c = uint32_t(i_sel);
        pop(2);
        return;
      }
      case PC_OP_LOOPIF: {
        if (x.time == 0) {  // loopif(c, a, b, 0) = if(c, a, b) (Sec. 6.1 rewrite)
          TNode y = x;
          node(x.ch[0]);
          size_t i_if = emit(X_IF);
          node(x.ch[1]);
          size_t i_else = emit(X_ELSE);
          node(x.ch[2]);
          size_t i_sel = emit(X_SEL);
          code[i_if].c = uint32_t(i_else + 1);
          code[i_else].c = uint32_t(i_sel);
          pop(2);
          (void)y;
          return;
        }
        ++n_loops;
        const uint32_t frame = uint32_t(nest);   // frame index; slot resolved later
        max_nest = std::max(max_nest, ++nest);
        const uint32_t n = uint32_t(x.time);
        const size_t i_loop = emit(X_LOOP, frame, n);
        size_t cond_pc = code.size();
        node(x.ch[0]);
        const TNode &th = T[x.ch[1]];
        const bool lit_then = th.op == PC_OP_REAL || th.op == PC_OP_BOOL || th.op == PC_OP_NAT;
        const uint32_t cop = code.back().opa & 0xffu;
        const bool one_fused = code.size() == cond_pc + 1 &&
                               (cop == X_LANY || (cop == X_LRED && ((code.back().opa >> 12) & 7u) != 0));
        if (lit_then && one_fused) {
          // whole loop in one instruction; the condition stays as a descriptor
          const uint32_t pidx = uint32_t(pool.size());
          pool.push_back(th.op == PC_OP_REAL ? float(th.val) : 0.f);
          if (th.op != PC_OP_REAL) std::memcpy(&pool.back(), &th.a, 4);
          code[i_loop].opa = X_LOOPANY | ((frame | (pidx << 8)) << 8);
          code[i_loop].c = uint32_t(cond_pc);
          pop();
          node(x.ch[2]);
          emit(X_LEND, frame);
          code[i_loop].e = uint32_t(code.size());
        } else if (lit_then) {
          // literal then-branch: test, latch and step in one instruction
          const uint32_t pidx = uint32_t(pool.size());
          pool.push_back(th.op == PC_OP_REAL ? float(th.val) : 0.f);
          if (th.op != PC_OP_REAL) std::memcpy(&pool.back(), &th.a, 4);
          const size_t i_step = emit(X_LSTEPK, frame | (pidx << 8), n, uint32_t(cond_pc));
          pop();
          code[i_loop].c = uint32_t(i_step);
          node(x.ch[2]);
          emit(X_LEND, frame);
          code[i_step].e = uint32_t(code.size());
        } else {
          size_t i_test = emit(X_LTEST, frame);
          pop();
          code[i_loop].c = uint32_t(i_test);
          node(x.ch[1]);
          emit(X_LLATCH, frame);
          pop();
          size_t i_next = emit(X_LNEXT, frame, n, uint32_t(cond_pc));
          node(x.ch[2]);
          emit(X_LEND, frame);
          code[i_test].c = uint32_t(i_next);
          code[i_next].e = uint32_t(code.size());
        }
        --nest;
        return;  // else-value popped and result pushed: net +1 as pushed by else
      }
      default: break;
    }
    if (try_fused(k)) return;
    // binary operators
    const TNode &l = T[x.ch[0]], &r = T[x.ch[1]];
    const bool real = l.ty == T_REAL && x.op != PC_OP_AND && x.op != PC_OP_OR;
    if (real && real_lit(r) && !real_lit(l)) {
      uint32_t xo = 0;
      switch (x.op) {
        case PC_OP_ADD: xo = X_ADDFK; break;
        case PC_OP_SUB: xo = X_SUBFK; break;
        case PC_OP_MULT: xo = X_MULFK; break;
        case PC_OP_DIV: xo = X_DIVFK; break;
        case PC_OP_MAX: xo = X_MAXFK; break;
        case PC_OP_MIN: xo = X_MINFK; break;
        case PC_OP_LT: xo = X_LTFK; break;
        case PC_OP_LE: xo = X_LEFK; break;
        case PC_OP_EQ: xo = X_EQFK; break;
      }
      if (xo) { node(x.ch[0]); imm(xo, float(r.val)); return; }
    }
    if (real && real_lit(l) && !real_lit(r)) {
      uint32_t xo = 0;
      switch (x.op) {
        case PC_OP_ADD: xo = X_ADDFK; break;
        case PC_OP_MULT: xo = X_MULFK; break;
        case PC_OP_MAX: xo = X_MAXFK; break;
        case PC_OP_MIN: xo = X_MINFK; break;
        case PC_OP_EQ: xo = X_EQFK; break;
        case PC_OP_SUB: xo = X_RSUBFK; break;
        case PC_OP_DIV: xo = X_RDIVFK; break;
        case PC_OP_LT: xo = X_RLTFK; break;
        case PC_OP_LE: xo = X_RLEFK; break;
      }
      if (xo) { node(x.ch[1]); imm(xo, float(l.val)); return; }
    }
    node(x.ch[0]);
    node(x.ch[1]);
    uint32_t xo = 0;
    if (x.op == PC_OP_AND) xo = X_AND;
    else if (x.op == PC_OP_OR) xo = X_OR;
    else if (x.op == PC_OP_EQ && l.ty == T_BOOL) xo = X_EQI;
    else if (real) {
      switch (x.op) {
        case PC_OP_ADD: xo = X_ADDF; break; case PC_OP_SUB: xo = X_SUBF; break;
        case PC_OP_MULT: xo = X_MULF; break; case PC_OP_DIV: xo = X_DIVF; break;
        case PC_OP_MAX: xo = X_MAXF; break; case PC_OP_MIN: xo = X_MINF; break;
        case PC_OP_LT: xo = X_LTF; break; case PC_OP_LE: xo = X_LEF; break;
        case PC_OP_EQ: xo = X_EQF; break;
      }
    } else {
      switch (x.op) {
        case PC_OP_ADD: xo = X_ADDI; break; case PC_OP_SUB: xo = X_SUBI; break;
        case PC_OP_MULT: xo = X_MULI; break;
        case PC_OP_MAX: xo = X_MAXI; break; case PC_OP_MIN: xo = X_MINI; break;
        case PC_OP_LT: xo = X_LTI; break; case PC_OP_LE: xo = X_LEI; break;
        case PC_OP_EQ: xo = X_EQI; break;
      }
    }
    emit(xo);
    pop();
  }

  // immediate form; fold a preceding MODEL into MODEL_MULK / MODEL_DIVK and
  // drop division by exactly 1.
  void imm(uint32_t xo, float k) {
    if (xo == X_DIVFK && k == 1.0f) return;
    if (xo == X_MULFK && k == 1.0f) return;
    XInsn &prev = code.back();
    if ((prev.opa & 0xff) == X_PAYOFF && xo == X_MULFK && prev.c == fbits(1.0f)) {
      prev.c = fbits(k);  // k * payoff(t): one instruction
      return;
    }
    if ((prev.opa & 0xff) == X_MODEL && (xo == X_MULFK || xo == X_DIVFK)) {
      prev.opa = (xo == X_MULFK ? X_MODEL_MULK : X_MODEL_DIVK) | (prev.opa & ~0xffu);
      prev.c = fbits(k);
      return;
    }
    emit(xo, 0, fbits(k));
  }
};

}  // namespace

pc_status compile_program(const uint32_t *words, size_t n_words, const double *consts,
                          size_t n_consts, const int32_t *tparams, size_t n_params,
                          int32_t p1, int32_t p2, bool bind_parties, Program &out,
                          std::string &err) {
  if (!words || n_words == 0) { err = "empty program"; return PC_EINVAL; }
  if (n_words > PC_MAX_PROGRAM) { err = "program exceeds PC_MAX_PROGRAM words"; return PC_ELIMIT; }
  if (n_consts > PC_MAX_CONSTS) { err = "too many constants"; return PC_ELIMIT; }
  if (n_params > PC_MAX_TPARAMS) { err = "too many template parameters"; return PC_ELIMIT; }
  if (n_consts && !consts) { err = "null consts"; return PC_EINVAL; }
  if (n_params && !tparams) { err = "null template_params"; return PC_EINVAL; }
  std::vector<TNode> T;
  std::vector<int32_t> st;
  Decoder D(words, n_words, tparams, n_params, err);
  while (D.i < n_words) {
    const uint32_t w = words[D.i++];
    const uint32_t op = w & 0xffu, A = w >> 8;
    TNode x;
    x.op = op;
    auto need = [&](int k) -> bool {
      if (int(st.size()) < k) { err = "stack underflow"; return false; }
      x.nch = k;
      for (int c = k - 1; c >= 0; --c) { x.ch[c] = st.back(); st.pop_back(); }
      return true;
    };
    pc_status s = PC_OK;
    switch (op) {
      case PC_OP_REAL:
        if (A >= n_consts) { err = "constant index out of range"; return PC_EBYTECODE; }
        if (!std::isfinite(consts[A])) { err = "constant not finite"; return PC_EBYTECODE; }
        x.val = consts[A];
        break;
      case PC_OP_BOOL:
        if (A > 1) { err = "bool literal must be 0 or 1"; return PC_EBYTECODE; }
        x.a = int32_t(A);
        break;
      case PC_OP_NAT: x.a = int32_t(A); break;
      case PC_OP_NOW: break;
      case PC_OP_TEXPR: s = D.time(1, x.time); break;
      case PC_OP_MODEL:
        if (A >= PC_MAX_UNDERLYINGS) { err = "label out of range"; return PC_EBYTECODE; }
        x.a = int32_t(A);
        s = D.time(0, x.time);
        break;
      case PC_OP_PAYOFF: {
        if (D.i + 2 > n_words) { err = "truncated payoff"; return PC_EBYTECODE; }
        int32_t q1 = int32_t(words[D.i]), q2 = int32_t(words[D.i + 1]);
        D.i += 2;
        s = D.time(1, x.time);
        if (bind_parties) x.sign = (q1 == p1 && q2 == p2) ? 1 : (q1 == p2 && q2 == p1) ? -1 : 0;
        else x.sign = 1;
        break;
      }
      case PC_OP_NEG: case PC_OP_NOT:
        if (!need(1)) return PC_EBYTECODE;
        break;
      case PC_OP_ADD: case PC_OP_SUB: case PC_OP_MULT: case PC_OP_DIV: case PC_OP_LT:
      case PC_OP_LE: case PC_OP_EQ: case PC_OP_AND: case PC_OP_OR: case PC_OP_MAX: case PC_OP_MIN:
        if (A) { err = "operator takes no operand"; return PC_EBYTECODE; }
        if (!need(2)) return PC_EBYTECODE;
        break;
      case PC_OP_IF:
        if (!need(3)) return PC_EBYTECODE;
        break;
      case PC_OP_LOOPIF:
        s = D.time(2, x.time);
        if (s == PC_OK && !need(3)) return PC_EBYTECODE;
        break;
      default:
        err = "bad opcode " + std::to_string(op);
        return PC_EBYTECODE;
    }
    if (s != PC_OK) return s;
    st.push_back(int32_t(T.size()));
    T.push_back(x);
  }
  if (st.size() != 1) { err = st.empty() ? "empty program" : "program leaves several values"; return PC_EBYTECODE; }
  pc_status s = typecheck(T, st[0], err);
  if (s != PC_OK) return s;
  Emitter E(T);
  E.node(st[0]);
  E.emit(X_END);
  const int stack_slots = E.max_depth + 1;  // slot 0 is the push sink of an empty stack
  if (stack_slots + LF_SLOTS * E.max_nest > PC_MAX_STACK) {
    err = "program needs a deeper stack than PC_MAX_STACK";
    return PC_ELIMIT;
  }
  // resolve loop frame indices to slot offsets after the operand slots
  for (XInsn &I : E.code) {
    uint32_t op = I.opa & 0xffu;
    if (op == X_LOOP || op == X_LTEST || op == X_LLATCH || op == X_LNEXT || op == X_LEND) {
      uint32_t f = I.opa >> 8;
      I.opa = op | (uint32_t(stack_slots + LF_SLOTS * f) << 8);
    } else if (op == X_LSTEPK || op == X_LOOPANY) {
      uint32_t f = (I.opa >> 8) & 0xffu, pidx = I.opa >> 16;
      I.opa = op | (uint32_t(stack_slots + LF_SLOTS * f) << 8) | (pidx << 16);
    }
  }
  if (E.pool.size() > 0xffff) { err = "too many fused-op constants"; return PC_ELIMIT; }
  if (stack_slots + LF_SLOTS * E.max_nest > 255) { err = "loop frames beyond slot 255"; return PC_ELIMIT; }
  out.pool = std::move(E.pool);
  out.code = std::move(E.code);
  out.frame_slots = stack_slots + LF_SLOTS * E.max_nest;
  out.info.n_nodes = int32_t(T.size());
  out.info.n_insn = int32_t(out.code.size());
  out.info.max_stack = out.frame_slots;
  out.info.result_is_real = 1;
  out.info.n_loops = E.n_loops;
  out.info.n_tparams_used = D.max_tp;
  return PC_OK;
}

pc_status analyse_program(const Program &p, int32_t t_now, int32_t n_dates, int32_t n_hist,
                          int32_t &win, std::string &err) {
  auto on_fail = [&](pc_status st, int64_t t, int64_t o) {
    if (st == PC_ELIMIT)
      err = "program too long to analyse (loop trip counts)";
    else
      err = "time " + std::to_string(t) + " is outside the model's grid (ordinal " + std::to_string(o) +
            ", grid " + std::to_string(-n_hist) + ".." + std::to_string(n_dates) + ")";
  };
  TimeWalk<decltype(on_fail)> walk{p.code.data(), t_now, n_dates, n_hist, on_fail};
  walk.run(0, p.code.size(), 0);
  if (walk.st != PC_OK) return walk.st;
  win = walk.window();
  return PC_OK;
}

// ---------------------------------------------------------------------------
// cutPayoff (Sec. 4.1) on the bytecode
// ---------------------------------------------------------------------------
// Every payoff(t, p1', p2') becomes if(t < now, 0, payoff(t, p1', p2')): in
// postfix, TEXPR t  NOW  LT  REAL 0.0  PAYOFF p1' p2' t  IF.  Every other
// instruction is copied; 0.0 is appended to the literals unless present.
pc_status cut_payoff(const uint32_t *w, size_t n, const double *consts, size_t n_consts,
                     std::vector<uint32_t> &out, std::vector<double> &out_consts, std::string &err) {
  out.clear();
  out_consts.assign(consts, consts + n_consts);
  uint32_t zero = uint32_t(n_consts);
  for (size_t k = 0; k < n_consts; ++k)
    if (consts[k] == 0.0 && !std::signbit(consts[k])) { zero = uint32_t(k); break; }
  bool zero_used = false;
  auto time_len = [&](size_t at, size_t &len) -> bool {
    if (at >= n) return false;
    const uint32_t c = w[at];
    if (c == 0 || c > 16 || at + 1 + c > n) return false;
    len = 1 + c;
    return true;
  };
  for (size_t i = 0; i < n;) {
    const uint32_t op = w[i] & 0xffu;
    size_t len = 1, tl = 0;
    switch (op) {
      case PC_OP_REAL: case PC_OP_BOOL: case PC_OP_NAT: case PC_OP_NOW:
      case PC_OP_NEG: case PC_OP_NOT: case PC_OP_ADD: case PC_OP_SUB: case PC_OP_MULT: case PC_OP_DIV:
      case PC_OP_LT: case PC_OP_LE: case PC_OP_EQ: case PC_OP_AND: case PC_OP_OR: case PC_OP_MAX:
      case PC_OP_MIN: case PC_OP_IF:
        break;
      case PC_OP_TEXPR: case PC_OP_MODEL: case PC_OP_LOOPIF:
        if (!time_len(i + 1, tl)) { err = "truncated time expression"; return PC_EBYTECODE; }
        len = 1 + tl;
        break;
      case PC_OP_PAYOFF: {
        if (!time_len(i + 3, tl)) { err = "truncated payoff"; return PC_EBYTECODE; }
        const uint32_t *t = w + i + 3;
        out.push_back(PC_OP_TEXPR);
        out.insert(out.end(), t, t + tl);
        out.push_back(PC_OP_NOW);
        out.push_back(PC_OP_LT);
        out.push_back(PC_OP_REAL | (zero << 8));
        zero_used = true;
        out.insert(out.end(), w + i, w + i + 3 + tl);
        out.push_back(PC_OP_IF);
        i += 3 + tl;
        continue;
      }
      default:
        err = "bad opcode " + std::to_string(op) + " at word " + std::to_string(i);
        return PC_EBYTECODE;
    }
    out.insert(out.end(), w + i, w + i + len);
    i += len;
  }
  if (zero_used && zero == n_consts) out_consts.push_back(0.0);
  return PC_OK;
}

// ---------------------------------------------------------------------------
// Text assembler
// ---------------------------------------------------------------------------
namespace {

struct Asm {
  std::vector<std::string> tok;
  size_t i = 0;
  std::vector<uint32_t> &w;
  std::vector<double> &k;
  std::map<uint64_t, uint32_t> kidx;
  std::string &err;

  Asm(const char *text, std::vector<uint32_t> &w_, std::vector<double> &k_, std::string &e)
      : w(w_), k(k_), err(e) {
    std::string s(text);
    std::string cur;
    bool comment = false;
    for (char ch : s) {
      if (comment) { if (ch == '\n') comment = false; continue; }
      if (ch == ';') { if (!cur.empty()) tok.push_back(cur); cur.clear(); comment = true; continue; }
      if (ch == '(' || ch == ')') {
        if (!cur.empty()) tok.push_back(cur);
        cur.clear();
        tok.push_back(std::string(1, ch));
      } else if (ch == ' ' || ch == '\t' || ch == '\n' || ch == '\r') {
        if (!cur.empty()) tok.push_back(cur);
        cur.clear();
      } else {
        cur += ch;
      }
    }
    if (!cur.empty()) tok.push_back(cur);
  }

  bool fail(const std::string &m) { err = m + " (token " + std::to_string(i) + ")"; return false; }
  bool more() const { return i < tok.size(); }
  const std::string &peek() { static std::string e; return more() ? tok[i] : e; }
  bool expect(const char *t) {
    if (!more() || tok[i] != t) return fail(std::string("expected '") + t + "'");
    ++i;
    return true;
  }
  bool integer(int64_t &v) {
    if (!more()) return fail("expected integer");
    const std::string &t = tok[i];
    char *end = nullptr;
    long long x = std::strtoll(t.c_str(), &end, 10);
    if (t.empty() || *end) return fail("bad integer '" + t + "'");
    v = x;
    ++i;
    return true;
  }
  // time expression -> list of term words
  bool time(std::vector<uint32_t> &terms) {
    if (!more()) return fail("expected time expression");
    if (tok[i] == "(") {
      ++i;
      if (!expect("tplus")) return false;
      if (!time(terms) || !time(terms)) return false;
      return expect(")");
    }
    if (tok[i][0] == '$') {
      char *end = nullptr;
      long v = std::strtol(tok[i].c_str() + 1, &end, 10);
      if (*end || v < 0 || v > 0x7fffffff) return fail("bad template variable");
      terms.push_back(0x80000000u | uint32_t(v));
      ++i;
      return true;
    }
    int64_t v;
    if (!integer(v)) return false;
    if (v < -(int64_t(1) << 30) || v >= (int64_t(1) << 30)) return fail("time literal out of range");
    terms.push_back(uint32_t(int32_t(v)) & 0x7fffffffu);
    return true;
  }
  bool emit_time() {
    std::vector<uint32_t> t;
    if (!time(t)) return false;
    if (t.size() > 16) return fail("time expression has more than 16 terms");
    w.push_back(uint32_t(t.size()));
    w.insert(w.end(), t.begin(), t.end());
    return true;
  }
  uint32_t konst(double v) {
    uint64_t bits;
    std::memcpy(&bits, &v, 8);
    auto it = kidx.find(bits);
    if (it != kidx.end()) return it->second;
    uint32_t id = uint32_t(k.size());
    k.push_back(v);
    kidx[bits] = id;
    return id;
  }
  bool expr() {
    if (!more()) return fail("unexpected end of text");
    std::string t = tok[i];
    if (t == "#t" || t == "#f") { ++i; w.push_back(PC_OP_BOOL | (uint32_t(t == "#t") << 8)); return true; }
    if (t != "(") {
      if (t.find_first_of(".eE") == std::string::npos || t[0] == '$') return fail("bad literal '" + t + "'");
      char *end = nullptr;
      double v = std::strtod(t.c_str(), &end);
      if (*end || !std::isfinite(v)) return fail("bad real literal '" + t + "'");
      ++i;
      uint32_t id = konst(v);
      if (id >= (1u << 24)) return fail("too many constants");
      w.push_back(PC_OP_REAL | (id << 8));
      return true;
    }
    ++i;
    if (!more()) return fail("unexpected end of text");
    std::string h = tok[i++];
    static const std::map<std::string, uint32_t> bin = {
        {"add", PC_OP_ADD}, {"sub", PC_OP_SUB}, {"mult", PC_OP_MULT}, {"div", PC_OP_DIV},
        {"lt", PC_OP_LT}, {"le", PC_OP_LE}, {"eq", PC_OP_EQ}, {"and", PC_OP_AND},
        {"or", PC_OP_OR}, {"max", PC_OP_MAX}, {"min", PC_OP_MIN}};
    if (h == "now") {
      w.push_back(PC_OP_NOW);
    } else if (h == "nat") {
      int64_t v;
      if (!integer(v)) return false;
      if (v < 0 || v >= (1 << 24)) return fail("nat literal out of range");
      w.push_back(PC_OP_NAT | (uint32_t(v) << 8));
    } else if (h == "texpr") {
      w.push_back(PC_OP_TEXPR);
      if (!emit_time()) return false;
    } else if (h == "model") {
      int64_t l;
      if (!integer(l)) return false;
      if (l < 0 || l >= PC_MAX_UNDERLYINGS) return fail("label out of range");
      w.push_back(PC_OP_MODEL | (uint32_t(l) << 8));
      if (!emit_time()) return false;
    } else if (h == "payoff") {
      std::vector<uint32_t> t;
      if (!time(t)) return false;
      int64_t q1, q2;
      if (!integer(q1) || !integer(q2)) return false;
      if (t.size() > 16) return fail("time expression has more than 16 terms");
      w.push_back(PC_OP_PAYOFF);
      w.push_back(uint32_t(int32_t(q1)));
      w.push_back(uint32_t(int32_t(q2)));
      w.push_back(uint32_t(t.size()));
      w.insert(w.end(), t.begin(), t.end());
    } else if (h == "neg" || h == "not") {
      if (!expr()) return false;
      w.push_back(h == "neg" ? PC_OP_NEG : PC_OP_NOT);
    } else if (bin.count(h)) {
      if (!expr() || !expr()) return false;
      w.push_back(bin.at(h));
    } else if (h == "if") {
      if (!expr() || !expr() || !expr()) return false;
      w.push_back(PC_OP_IF);
    } else if (h == "loopif") {
      if (!expr() || !expr() || !expr()) return false;
      w.push_back(PC_OP_LOOPIF);
      if (!emit_time()) return false;
    } else {
      return fail("unknown construct '" + h + "'");
    }
    return expect(")");
  }
};

}  // namespace

pc_status assemble_text(const char *text, std::vector<uint32_t> &words,
                        std::vector<double> &consts, std::string &err) {
  words.clear();
  consts.clear();
  Asm a(text, words, consts, err);
  if (!a.expr()) return PC_ESYNTAX;
  if (a.more()) { err = "trailing tokens after the expression"; return PC_ESYNTAX; }
  return PC_OK;
}

}  // namespace pc
