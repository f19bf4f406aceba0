// pc_jit.cpp -- run-time specialised pricing kernels.
//
// The paper compiles each contract to a payoff function of its own (Sec. 6:
// Futhark code per instrument).  The engine's default kernel interprets the
// executable program instead, which costs a dispatch per instruction.  Here
// the program is turned into straight-line CUDA: one labelled block per
// instruction, each the interpreter's case for that opcode (the text of
// pc_ops.inc, split per opcode at build time), with NEXT / JUMP_* as gotos
// between the blocks.  The block bodies are the
// interpreter's own text, so both evaluators compute the same operations in
// the same order.  NVRTC compiles the module for the device the context
// runs on; the kernel is price_tiles (pc_price.cuh) with this evaluator.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include <nvrtc.h>

#include "pc_handles.h"
#include "pc_internal.h"
#include "pc_cv_types.h"
#include "pc_jit_headers.inc"

using namespace pc;

namespace {

std::string hex(uint32_t v) {
  char b[16];
  std::snprintf(b, sizeof(b), "0x%08xu", v);
  return b;
}

// The interpreter's case for an opcode (pc_ops.inc, split by the build);
// unknown opcodes take the default case (return), as in the interpreter.
const char *case_text(uint32_t op) {
  return op < uint32_t(kJitCaseCount) ? kJitCase[op] : kJitCase[0];
}

std::string insn_literal(const XInsn &I) {
  return "make_uint4(" + hex(I.opa) + ", " + hex(I.b) + ", " + hex(I.c) + ", " + hex(I.e) + ")";
}

// Above this many reading instructions a program whose stack depths are
// not known calls the date generator out of line.
constexpr int kInlineDateSites = 12;
// Above this many reading instructions the re-entry switch of the shared
// generator makes NVRTC's time grow faster than the program (100 terms of
// a two-asset average: 13 s shared, 3.2 s out of line): call it out of line.
constexpr int kSharedDateSites = 64;
// The tangent date generator (S and X windows) is about twice the size of
// the pricing one: inlined at up to this many reading instructions.
constexpr int kInlineTangentDateSites = 6;

// Instructions that read simulated dates (and may have to generate them).
bool reads_dates(const XInsn &I) {
  const uint32_t op = I.opa & 0xffu;
  return op == X_MODEL || op == X_MODEL_MULK || op == X_MODEL_DIVK || op == X_LRED || op == X_LANY;
}

int date_sites(const Program &p) {
  int n = 0;
  for (const XInsn &I : p.code) n += reads_dates(I);
  return n;
}

// The evaluator's operand-stack pointer (sp) before each instruction, from
// every opcode's effect on each of its exits (the cases of pc_ops.inc):
// -1 for instructions no path reaches.  False when an opcode has no known
// effect, a depth leaves [0, frame_slots), or two paths meet with different
// depths -- the program is then specialised without re-entry points.
bool stack_depths(const Program &p, std::vector<int> &sp_at) {
  const int n = int(p.code.size());
  sp_at.assign(size_t(n), -1);
  if (n == 0) return false;
  std::vector<int> work;
  bool ok = true;
  auto flow = [&](uint32_t t, int v) {
    if (t >= uint32_t(n) || v < 0 || v >= std::max(1, int(p.frame_slots))) {
      ok = false;
      return;
    }
    if (sp_at[t] < 0) {
      sp_at[t] = v;
      work.push_back(int(t));
    } else if (sp_at[t] != v) {
      ok = false;
    }
  };
  flow(0, 0);
  while (ok && !work.empty()) {
    const int i = work.back();
    work.pop_back();
    const XInsn &I = p.code[size_t(i)];
    const int s = sp_at[size_t(i)];
    const uint32_t nx = uint32_t(i + 1);
    switch (I.opa & 0xffu) {
      case X_END: break;
      case X_CONST: case X_MODEL: case X_PAYOFF: case X_TIME: case X_NOW: case X_MODEL_MULK:
      case X_MODEL_DIVK: case X_LRED: case X_LANY:
        flow(nx, s + 1);
        break;
      case X_NEGF: case X_NOT: case X_ADDFK: case X_SUBFK: case X_MULFK: case X_DIVFK: case X_MAXFK:
      case X_MINFK: case X_LTFK: case X_LEFK: case X_EQFK: case X_RSUBFK: case X_RDIVFK: case X_RLTFK:
      case X_RLEFK: case X_LOOP: case X_LEND:
        flow(nx, s);
        break;
      case X_ADDF: case X_SUBF: case X_MULF: case X_DIVF: case X_MAXF: case X_MINF: case X_LTF: case X_LEF:
      case X_EQF: case X_ADDI: case X_SUBI: case X_MULI: case X_MAXI: case X_MINI: case X_LTI: case X_LEI:
      case X_EQI: case X_AND: case X_OR: case X_LLATCH:
        flow(nx, s - 1);
        break;
      case X_SEL: flow(nx, s - 2); break;
      case X_IF: case X_ELSE:  // NEXT, or push a placeholder and JUMP_Z
        flow(nx, s);
        flow(I.c, s + 1);
        break;
      case X_LTEST:  // pop; NEXT or JUMP_Z
        flow(nx, s - 1);
        flow(I.c, s - 1);
        break;
      case X_LSTEPK:  // pop; push the result and JUMP_W, NEXT, or JUMP_Z
        flow(I.e, s);
        flow(nx, s - 1);
        flow(I.c, s - 1);
        break;
      case X_LNEXT:
        flow(I.e, s + 1);
        flow(nx, s);
        flow(I.c, s);
        break;
      case X_LOOPANY:  // push the result and JUMP_W, or JUMP_2 (pc + 1 is a descriptor)
        flow(I.e, s + 1);
        flow(uint32_t(i + 2), s);
        break;
      default: ok = false; break;
    }
  }
  return ok;
}

// Straight-line tangent evaluator (pc_jit_greeks around greeks_tiles; the
// per-path triples written out with kJitGreeks + 1): each instruction is
// the interpreter's case for its constant opcode and fields, followed by a
// jump to whichever of its possible successors the case left in pc.  The
// operand stack of value-with-tangents stays in shared memory, as in the
// interpreter.  Beyond kInlineTangentDateSites reading instructions they
// call one out-of-line copy of the date generator.
// The adjoint evaluator straight-line over the program (each instruction's
// block includes pc_adjoint_ops.inc with the instruction as a constant),
// and pc_jit_adjoint: adjoint_tiles around it.  The date generator (with
// the X window) is inlined at each reading instruction: programs with more
// than kInlineTangentDateSites of them are not specialised (adjoint_eligible).
std::string generate_adjoint(const Program &p, int d, bool write) {
  std::ostringstream o;
  const size_t n = p.code.size();
  o << "#include \"pc_adjoint.cuh\"\n"
    << "namespace pc {\n"
    << "namespace {\n"
    << "constexpr int D = " << d << ";\n"
    << "__device__ __forceinline__ float2 jit_eval_adjoint(const uint4 *P, const float *pool, float2 *R,\n"
    << "    const PriceArgs &a, const Rng2 &g, bool live0, bool live1, const float (&Bm)[D * D],\n"
    << "    const float (&S0)[D], const float (&Lm)[D * D], Tape &T, int &res) {\n"
    << "#include \"pc_adjoint_state.inc\"\n"
    << "  goto L0;\n";
  for (size_t i = 0; i < n; ++i) {
    const XInsn &I = p.code[i];
    o << "L" << i << ": {\n"
      << "  pc = " << i << ";\n"
      << "  const uint4 I = " << insn_literal(I) << ";\n"
      << "  const uint32_t op = " << hex(I.opa & 0xffu) << ";\n"
      << "  const float kk = __uint_as_float(" << hex(I.b) << ");\n"
      << "#include \"pc_adjoint_ops.inc\"\n";
    std::vector<uint32_t> next = {uint32_t(i + 1), I.c, I.e, uint32_t(i + 2)};
    for (size_t j = 0; j < next.size(); ++j) {
      bool seen = false;
      for (size_t q = 0; q < j; ++q) seen = seen || next[q] == next[j];
      if (!seen && next[j] < n) o << "  if (pc == " << next[j] << ") goto L" << next[j] << ";\n";
    }
    o << "  res = tid;\n"
      << "  return tos;\n"
      << "}\n";
  }
  o << "}\n"
    << "}  // namespace\n"
    << "}  // namespace pc\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << kBlock
    << ") pc_jit_adjoint(const __grid_constant__ pc::PriceArgs a, const pc::TapeArgs t) {\n"
    << "  pc::adjoint_tiles<pc::D, " << (write ? "true" : "false") << ">(a, t, [&](const uint4 *P, const float *pool,\n"
    << "      float2 *R, const pc::Rng2 &g, bool live0, bool live1, const float (&Bm)[pc::D * pc::D],\n"
    << "      const float (&S0)[pc::D], const float (&Lm)[pc::D * pc::D], pc::Tape &T, int &res) {\n"
    << "    return pc::jit_eval_adjoint(P, pool, R, a, g, live0, live1, Bm, S0, Lm, T, res); });\n"
    << "}\n";
  return o.str();
}

std::string generate_greeks(const Program &p, int d, bool write) {
  std::ostringstream o;
  const size_t n = p.code.size();
  if (date_sites(p) > kInlineTangentDateSites) o << "#define PC_JIT_OUTLINE_DATES 1\n";
  o << "#include \"pc_greeks.cuh\"\n"
    << "namespace pc {\n"
    << "namespace {\n"
    << "constexpr int D = " << d << ";\n"
    << "__device__ __forceinline__ TV jit_eval_greeks(const uint4 *P, const float *pool, float2 *R,\n"
    << "    const PriceArgs &a, const Rng2 &g, bool live0, bool live1, const float (&Bm)[D * D],\n"
    << "    const float (&S0)[D], const float (&Lm)[D * D], int gl, float sig_g) {\n"
    << "#include \"pc_greeks_state.inc\"\n"
    << "  goto L0;\n";
  for (size_t i = 0; i < n; ++i) {
    const XInsn &I = p.code[i];
    o << "L" << i << ": {\n"
      << "  pc = " << i << ";\n"
      << "  const uint4 I = " << insn_literal(I) << ";\n"
      << "  const uint32_t op = " << hex(I.opa & 0xffu) << ";\n"
      << "  const float kk = __uint_as_float(" << hex(I.b) << ");\n"
      << "#include \"pc_greeks_ops.inc\"\n";
    std::vector<uint32_t> next = {uint32_t(i + 1), I.c, I.e, uint32_t(i + 2)};
    for (size_t j = 0; j < next.size(); ++j) {
      bool seen = false;
      for (size_t q = 0; q < j; ++q) seen = seen || next[q] == next[j];
      if (!seen && next[j] < n) o << "  if (pc == " << next[j] << ") goto L" << next[j] << ";\n";
    }
    o << "  return tos;\n"
      << "}\n";
  }
  o << "}\n"
    << "}  // namespace\n"
    << "}  // namespace pc\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << kBlock << ") pc_jit_greeks(const __grid_constant__ pc::PriceArgs a) {\n"
    << "  pc::greeks_tiles<pc::D, " << (write ? "true" : "false") << ">(a, [&](const uint4 *P, const float *pool,\n"
    << "      float2 *R, const pc::Rng2 &g, bool live0, bool live1, const float (&Bm)[pc::D * pc::D],\n"
    << "      const float (&S0)[pc::D], const float (&Lm)[pc::D * pc::D], int gl, float sig_g) {\n"
    << "    return pc::jit_eval_greeks(P, pool, R, a, g, live0, live1, Bm, S0, Lm, gl, sig_g); });\n"
    << "}\n";
  return o.str();
}

// Straight-line evaluator for the program and d underlyings, and the kernel
// of `kind` around it: pc_jit_price (price_tiles; per-path payoffs written
// out with kJitPriceWrite, the window of dates in HBM with kJitHbm) or
// pc_jit_cv (cv_tiles with mode kind - kJitCv).
// With two or more reading instructions and known stack depths, the date
// generator has one copy: a reading instruction that needs dates jumps to
// it and it jumps back to the top of that instruction, restoring the
// static stack pointer there (so the operand stack stays in registers).
// Otherwise the generator is inlined at each reading instruction (out of
// line beyond kInlineDateSites of them).
std::string generate(const Program &p, int d, int kind) {
  if (kind >= kJitAdjoint) return generate_adjoint(p, d, (kind & 1) != 0);
  if (kind >= kJitGreeks) return generate_greeks(p, d, (kind & 1) != 0);
  std::ostringstream o;
  const size_t n = p.code.size();
  std::vector<int> sp_at;
  const bool shared = date_sites(p) >= 2 && date_sites(p) <= kSharedDateSites && stack_depths(p, sp_at);
  // without re-entry points, many reading instructions call one
  // out-of-line copy instead of inlining the generator at each
  if (!shared && date_sites(p) > kInlineDateSites) o << "#define PC_JIT_OUTLINE_DATES 1\n";
  // a program that reads no date behind the frontier keeps that date's S in
  // registers instead of a shared-memory window
  if ((kind < kJitCv && (kind & kJitWinRegs)) || (kind >= kJitCv && ((kind - kJitCv) & kCvWinRegs)))
    o << "#define PC_WIN_REGS 1\n";
  // four paths a lane: the per-op and per-instruction control serves twice
  // the paths
  const bool pairs2 = kind < kJitCv && (kind & kJitPairs2);
  if (pairs2) o << "#define PC_PAIRS 2\n";
  o << "#include \"pc_price.cuh\"\n";
  if (kind >= kJitCv) o << "#include \"pc_cv.cuh\"\n";
  o
    << "namespace pc {\n"
    << "namespace {\n"
    << "constexpr int D = " << d << ";\n"
    << "constexpr bool GW = " << (kind < kJitCv && (kind & kJitHbm) ? "true" : "false") << ";\n"
    << "#define PC_JIT_STACK_SLOTS " << std::max(1, int(p.frame_slots)) << "\n"
    << "template <class PcHook = NoDateHook>\n"
    << "__device__ __forceinline__ PV jit_eval(const uint4 *P, const float *pool, float2 *R,\n"
    << (pairs2 ? "    const PriceArgs &a, const RngH<2> &g, const bool (&live_)[kPL], const float (&Bm)[D * D],\n"
               : "    const PriceArgs &a, const Rng2 &g, bool live0, bool live1, const float (&Bm)[D * D],\n")
    << "    const float (&S0)[D], int *frontier = nullptr, PcHook *hook_ = nullptr) {\n"
    << "#include \"pc_eval_state.inc\"\n"
    << "  (void)pc;\n";
  if (shared) {
    o << "  int need_ = 0, resume_ = -1;\n"
      << "  goto L0;\n"
      << "PC_GEN:\n"
      << "  while (ps.f < need_) GEN_DATE(ps.f + 1);\n"
      << "  switch (resume_) {\n";
    for (size_t i = 0; i < n; ++i)
      if (reads_dates(p.code[i]) && sp_at[i] >= 0)
        o << "    case " << i << ": sp = " << sp_at[i] << "; goto L" << i << ";\n";
    o << "    default: return tos;\n"
      << "  }\n";
  }
  for (size_t i = 0; i < n; ++i) {
    const XInsn &I = p.code[i];
    const size_t nx = i + 1 < n ? i + 1 : i;
    auto lbl = [&](size_t t) { return "L" + std::to_string(t < n ? t : n - 1); };
    o << lbl(i) << ": {\n"
      << "#define NEXT { goto " << lbl(nx) << "; }\n"
      << "#define JUMP_Z { goto " << lbl(I.c) << "; }\n"
      << "#define JUMP_W { goto " << lbl(I.e) << "; }\n"
      << "#define JUMP_2 { goto " << lbl(i + 2) << "; }\n"
      << "#define NEXT_INSN " << (i + 1 < n ? insn_literal(p.code[i + 1]) : insn_literal(I)) << "\n";
    if (shared && reads_dates(I) && sp_at[i] >= 0)
      o << "#define ENSURE(o) { if ((o) > m.n || (o) < -m.n_hist) { atomicOr(a.status, 1); "
           "(o) = (o) > m.n ? m.n : -m.n_hist; } if (ps.f < (o)) { need_ = (o); resume_ = "
        << i << "; goto PC_GEN; } }\n";
    else
      o << "#define ENSURE(o) ensure(o)\n";
    o << "  const uint4 I = " << insn_literal(I) << ";\n"
      << "  {\n" << case_text(I.opa & 0xffu) << "  }\n"
      << "#undef NEXT\n#undef JUMP_Z\n#undef JUMP_W\n#undef JUMP_2\n#undef NEXT_INSN\n#undef ENSURE\n"
      << "}\n";
  }
  o << "  return tos;\n"
    << "#undef PUSH\n#undef STK\n#undef BINF\n#undef BINI\n#undef IMM\n#undef GEN_DATE\n"
    << "}\n"
    << "}  // namespace\n"
    << "}  // namespace pc\n";
  if (kind >= kJitCv) {
    // the register bound (PC_MIN_BLOCKS resident blocks) is passed by the
    // launcher
    const bool gamma = ((kind - kJitCv) & kCvGamma) != 0;
    o << "#ifndef PC_MIN_BLOCKS\n#define PC_MIN_BLOCKS " << kJitCvMinBlocks << "\n#endif\n"
      << "extern \"C\" __global__ void __launch_bounds__(" << kBlock
      << ", PC_MIN_BLOCKS) pc_jit_cv(const __grid_constant__ pc::PriceArgs a,\n"
      << "    const __grid_constant__ pc::CvArgs c) {\n"
      << "  using Hook = pc::CvOnline<pc::D, " << (gamma ? "true" : "false") << ">;\n"
      << "  pc::cv_tiles<pc::D, " << ((kind - kJitCv) & 7) << ">(a, c, [&](const uint4 *P, const float *pool, float2 *R,\n"
      << "      const pc::Rng2 &g, bool live0, bool live1, const float (&Bm)[pc::D * pc::D],\n"
      << "      const float (&S0)[pc::D], Hook *hook) {\n"
      << "    return pc::jit_eval<Hook>(P, pool, R, a, g, live0, live1, Bm, S0, nullptr, hook); });\n"
      << "}\n";
    return o.str();
  }
  // resident 128-thread blocks per SM the register bound is set for
  // (PC_MIN_BLOCKS, passed by the launcher: 7, <= 72 registers, unless the
  // launch's shared memory already allows fewer, whose bound then leaves the
  // kernel the registers those blocks can have)
  o << "#ifndef PC_MIN_BLOCKS\n#define PC_MIN_BLOCKS " << kJitMinBlocks << "\n#endif\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << kBlock << ", PC_MIN_BLOCKS) pc_jit_price(const __grid_constant__ pc::PriceArgs a) {\n";
  if (pairs2)
    o << "  pc::price_tiles2<pc::D, " << (kind & kJitPriceWrite ? "true" : "false") << ">(a, [&](const uint4 *P, const float *pool,\n"
      << "      float2 *R, const pc::RngH<2> &g, const bool (&live)[4], const float (&Bm)[pc::D * pc::D],\n"
      << "      const float (&S0)[pc::D]) { return pc::jit_eval(P, pool, R, a, g, live, Bm, S0); });\n";
  else
    o << "  pc::price_tiles<pc::D, " << (kind & kJitPriceWrite ? "true" : "false") << ">(a, [&](const uint4 *P, const float *pool,\n"
      << "      float2 *R, const pc::Rng2 &g, bool live0, bool live1, const float (&Bm)[pc::D * pc::D],\n"
      << "      const float (&S0)[pc::D]) { return pc::jit_eval(P, pool, R, a, g, live0, live1, Bm, S0); });\n";
  o << "}\n";
  return o.str();
}

pc_status nvrtc_fail(nvrtcResult r, nvrtcProgram prog, const char *what) {
  std::string msg = std::string(what) + ": " + nvrtcGetErrorString(r);
  size_t n = 0;
  if (prog && nvrtcGetProgramLogSize(prog, &n) == NVRTC_SUCCESS && n > 1) {
    std::string log(n, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    msg += "\n" + log.substr(0, 4000);
  }
  return fail(PC_ECUDA, msg);
}

// NVRTC: the generated source and the embedded device headers to a cubin
// for `arch` (e.g. "sm_103a").
pc_status to_cubin(const Program &p, int d, int kind, int block, int min_blocks, const std::string &arch,
                   std::vector<char> &cubin) {
  const std::string src = generate(p, d, kind);
  nvrtcProgram prog = nullptr;
  nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "pc_jit.cu", kJitHeaderCount, kJitHeaderSrcs,
                                     kJitHeaderNames);
  if (r != NVRTC_SUCCESS) return nvrtc_fail(r, nullptr, "run-time compiler");
  const std::string a = "-arch=" + arch;
  const std::string stride = "-DPC_SLOT_STRIDE=" + std::to_string(block);
  const std::string bound = "-DPC_MIN_BLOCKS=" + std::to_string(min_blocks > 0 ? min_blocks : kJitMinBlocks);
  const char *opts[] = {a.c_str(), "-std=c++17", "-default-device", "-DPC_JIT", stride.c_str(), bound.c_str()};
  r = nvrtcCompileProgram(prog, 6, opts);
  if (r != NVRTC_SUCCESS) {
    pc_status s = nvrtc_fail(r, prog, "run-time compilation");
    nvrtcDestroyProgram(&prog);
    return s;
  }
  size_t n = 0;
  r = nvrtcGetCUBINSize(prog, &n);
  cubin.assign(n, 0);
  if (r == NVRTC_SUCCESS) r = nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  if (r != NVRTC_SUCCESS) return nvrtc_fail(r, nullptr, "cubin");
  return PC_OK;
}

pc_status compile(const Program &p, int d, int kind, int block, int min_blocks, int device, cudaLibrary_t &lib,
                  cudaKernel_t &kern) {
  cudaDeviceProp prop{};
  CU(cudaGetDeviceProperties(&prop, device), "device properties");
  std::vector<char> cubin;
  pc_status s = to_cubin(p, d, kind, block, min_blocks,
                         "sm_" + std::to_string(prop.major) + std::to_string(prop.minor) + "a", cubin);
  if (s != PC_OK) return s;
  CU(cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0), "module load");
  cudaError_t e = cudaLibraryGetKernel(&kern, lib, kind >= kJitAdjoint ? "pc_jit_adjoint"
                                                    : kind >= kJitGreeks ? "pc_jit_greeks"
                                                    : kind >= kJitCv ? "pc_jit_cv" : "pc_jit_price");
  if (e != cudaSuccess) {
    cudaLibraryUnload(lib);
    lib = nullptr;
    kern = nullptr;
    return cuda_fail(e, "kernel lookup");
  }
  return PC_OK;
}

}  // namespace

namespace pc {

bool jit_eligible(const pc_contract *k) { return k->prog.code.size() <= size_t(PC_JIT_MAX_INSNS); }

bool adjoint_jit_eligible(const pc_contract *k) {
  return jit_eligible(k) && date_sites(k->prog) <= kInlineTangentDateSites;
}

pc_status jit_kernel(const pc_contract *k, int d, int kind, int block, cudaKernel_t &out, int min_blocks) {
  // the program's words: code, then pool bits
  std::vector<uint32_t> words;
  words.reserve(k->prog.code.size() * 4 + k->prog.pool.size());
  for (const XInsn &I : k->prog.code) {
    words.push_back(I.opa);
    words.push_back(I.b);
    words.push_back(I.c);
    words.push_back(I.e);
  }
  for (float f : k->prog.pool) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    words.push_back(u);
  }
  uint64_t h = 1469598103934665603ull;  // FNV-1a
  for (uint32_t w : words)
    for (int b = 0; b < 4; ++b) h = (h ^ ((w >> (8 * b)) & 0xffu)) * 1099511628211ull;
  pc_ctx *c = k->ctx;
  std::lock_guard<std::mutex> g(c->jit_mu);
  auto range = c->jit_cache.equal_range(h);
  for (auto it = range.first; it != range.second; ++it) {
    const JitEntry &E = it->second;
    if (E.d == d && E.kind == kind && E.block == block && E.min_blocks == min_blocks && E.program == words) {
      out = E.kernel;
      return PC_OK;
    }
  }
  JitEntry E;
  E.program = words;
  E.d = d;
  E.kind = kind;
  E.block = block;
  E.min_blocks = min_blocks;
  pc_status s = compile(k->prog, d, kind, block, min_blocks, c->device, E.lib, E.kernel);
  if (s != PC_OK) return s;
  out = E.kernel;
  c->jit_cache.emplace(h, std::move(E));
  return PC_OK;
}

namespace {
const char *jit_entry_name(int kind) {
  return kind >= kJitAdjoint ? "pc_jit_adjoint" : kind >= kJitGreeks ? "pc_jit_greeks"
         : kind >= kJitCv ? "pc_jit_cv" : "pc_jit_price";
}

std::vector<uint32_t> program_words(const Program &p) {
  std::vector<uint32_t> words;
  words.reserve(p.code.size() * 4 + p.pool.size());
  for (const XInsn &I : p.code) {
    words.push_back(I.opa);
    words.push_back(I.b);
    words.push_back(I.c);
    words.push_back(I.e);
  }
  for (float f : p.pool) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    words.push_back(u);
  }
  return words;
}
}  // namespace

pc_status jit_compile_many(pc_ctx *c, const std::vector<JitRequest> &reqs) {
  // the requests not yet in the context's cache (each once)
  struct Miss {
    const JitRequest *r;
    std::vector<uint32_t> words;
    uint64_t h;
    std::vector<char> cubin;
    pc_status s = PC_OK;
  };
  std::vector<Miss> miss;
  {
    std::lock_guard<std::mutex> g(c->jit_mu);
    for (const JitRequest &r : reqs) {
      Miss m;
      m.r = &r;
      m.words = program_words(r.k->prog);
      uint64_t h = 1469598103934665603ull;  // FNV-1a, as jit_kernel
      for (uint32_t w : m.words)
        for (int b = 0; b < 4; ++b) h = (h ^ ((w >> (8 * b)) & 0xffu)) * 1099511628211ull;
      m.h = h;
      bool have = false;
      auto range = c->jit_cache.equal_range(h);
      for (auto it = range.first; it != range.second && !have; ++it) {
        const JitEntry &E = it->second;
        have = E.d == r.d && E.kind == r.kind && E.block == r.block && E.min_blocks == r.min_blocks &&
               E.program == m.words;
      }
      for (const Miss &o : miss)
        have = have || (o.h == h && o.r->d == r.d && o.r->kind == r.kind && o.r->block == r.block &&
                         o.r->min_blocks == r.min_blocks && o.words == m.words);
      if (!have) miss.push_back(std::move(m));
    }
  }
  if (miss.empty()) return PC_OK;
  cudaDeviceProp prop{};
  CU(cudaGetDeviceProperties(&prop, c->device), "device properties");
  const std::string arch = "sm_" + std::to_string(prop.major) + std::to_string(prop.minor) + "a";
  // NVRTC on the host's cores, one program per thread at a time
  std::atomic<size_t> next{0};
  auto work = [&]() {
    for (size_t i = next++; i < miss.size(); i = next++) {
      const JitRequest &r = *miss[i].r;
      miss[i].s = to_cubin(r.k->prog, r.d, r.kind, r.block, r.min_blocks, arch, miss[i].cubin);
    }
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>(miss.size(), std::min<unsigned>(hw, 32u));
  std::vector<std::thread> pool;
  for (size_t t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (std::thread &t : pool) t.join();
  std::lock_guard<std::mutex> g(c->jit_mu);
  for (Miss &m : miss) {
    if (m.s != PC_OK) return m.s;
    JitEntry E;
    E.program = m.words;
    E.d = m.r->d;
    E.kind = m.r->kind;
    E.block = m.r->block;
    E.min_blocks = m.r->min_blocks;
    CU(cudaLibraryLoadData(&E.lib, m.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0), "module load");
    cudaError_t e = cudaLibraryGetKernel(&E.kernel, E.lib, jit_entry_name(E.kind));
    if (e != cudaSuccess) {
      cudaLibraryUnload(E.lib);
      return cuda_fail(e, "kernel lookup");
    }
    c->jit_cache.emplace(m.h, std::move(E));
  }
  return PC_OK;
}

void jit_release(pc_ctx *c) {
  std::lock_guard<std::mutex> g(c->jit_mu);
  for (auto &kv : c->jit_cache)
    if (kv.second.lib) cudaLibraryUnload(kv.second.lib);
  c->jit_cache.clear();
}

}  // namespace pc

extern "C" pc_status pc_debug_jit_compile(const uint32_t *bytecode, size_t n_words, const double *consts,
                                          size_t n_consts, const int32_t *tparams, size_t n_params,
                                          int32_t p1, int32_t p2, int32_t d, int32_t kind,
                                          size_t *cubin_bytes) {
  if (!cubin_bytes) return fail(PC_EINVAL, "null output");
  if (d < 1 || d > PC_MAX_UNDERLYINGS) return fail(PC_EINVAL, "d must be 1..4");
  const int cvm = (kind - kJitCv) & 7;  // mode bits, with or without kCvWinRegs
  const bool cv_kind = kind >= kJitCv && kind < kJitCv + 16 && cvm != kCvWrite && cvm != (kCvWrite | kCvPilot) &&
                       cvm != (kCvWrite | kCvPilot | kCvGamma);
  const bool greeks_kind = kind == kJitGreeks || kind == kJitGreeks + 1 || kind == kJitAdjoint ||
                           kind == kJitAdjoint + 1;
  const bool price_kind = kind >= 0 && kind <= (kJitPriceWrite | kJitHbm | kJitWinRegs | kJitPairs2) &&
                          (!(kind & kJitPairs2) || (kind & (kJitWinRegs | kJitHbm)) == kJitWinRegs);
  if (!price_kind && !cv_kind && !greeks_kind)
    return fail(PC_EINVAL, "unknown kernel kind");
  if (cv_kind && d > kCvMaxD) return fail(PC_EINVAL, "control-variate kernels take d <= 3");
  Program p;
  std::string err;
  pc_status s = compile_program(bytecode, n_words, consts, n_consts, tparams, n_params, p1, p2, true, p, err);
  if (s != PC_OK) return fail(s, err);
  std::vector<char> cubin;
  s = to_cubin(p, d, kind, kBlock, 0, "sm_103a", cubin);
  if (s != PC_OK) return s;
  *cubin_bytes = cubin.size();
  return PC_OK;
}

extern "C" pc_status pc_debug_jit_source(const uint32_t *bytecode, size_t n_words, const double *consts,
                                         size_t n_consts, const int32_t *tparams, size_t n_params,
                                         int32_t p1, int32_t p2, int32_t d, int32_t kind, char *out,
                                         size_t cap, size_t *len) {
  if (!len) return fail(PC_EINVAL, "null output");
  if (d < 1 || d > PC_MAX_UNDERLYINGS) return fail(PC_EINVAL, "d must be 1..4");
  const bool known = (kind >= 0 && kind <= (kJitPriceWrite | kJitHbm | kJitWinRegs | kJitPairs2) &&
                      (!(kind & kJitPairs2) || (kind & (kJitWinRegs | kJitHbm)) == kJitWinRegs)) ||
                     (kind >= kJitCv && kind < kJitCv + 16) ||
                     kind == kJitGreeks || kind == kJitGreeks + 1 || kind == kJitAdjoint || kind == kJitAdjoint + 1;
  if (!known) return fail(PC_EINVAL, "unknown kernel kind");
  Program p;
  std::string err;
  pc_status s = compile_program(bytecode, n_words, consts, n_consts, tparams, n_params, p1, p2, true, p, err);
  if (s != PC_OK) return fail(s, err);
  const std::string src = generate(p, d, kind);
  *len = src.size();
  if (out && cap > src.size()) std::memcpy(out, src.c_str(), src.size() + 1);
  return PC_OK;
}
