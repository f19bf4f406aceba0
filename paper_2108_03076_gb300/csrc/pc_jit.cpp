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
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include <nvrtc.h>

#include "pc_handles.h"
#include "pc_internal.h"
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

// Instructions that read simulated dates (and may have to generate them);
// above this many, the date generator is called out of line instead of
// being inlined at each of them.
constexpr int kInlineDateSites = 12;

int date_sites(const Program &p) {
  int n = 0;
  for (const XInsn &I : p.code) {
    const uint32_t op = I.opa & 0xffu;
    n += op == X_MODEL || op == X_MODEL_MULK || op == X_MODEL_DIVK || op == X_LRED || op == X_LANY;
  }
  return n;
}

// Straight-line evaluator for the program and d underlyings, and the
// pricing kernel around it (per-path payoffs written out when `write`).
std::string generate(const Program &p, int d, bool write) {
  std::ostringstream o;
  const size_t n = p.code.size();
  if (date_sites(p) > kInlineDateSites) o << "#define PC_JIT_OUTLINE_DATES 1\n";
  o << "#include \"pc_price.cuh\"\n"
    << "namespace pc {\n"
    << "namespace {\n"
    << "constexpr int D = " << d << ";\n"
    << "constexpr bool GW = false;\n"
    << "#define PC_JIT_STACK_SLOTS " << std::max(1, int(p.frame_slots)) << "\n"
    << "__device__ __forceinline__ float2 jit_eval(const uint4 *P, const float *pool, float2 *R,\n"
    << "    const PriceArgs &a, const Rng2 &g, bool live0, bool live1, const float (&Bm)[D * D],\n"
    << "    const float (&S0)[D], int *frontier = nullptr) {\n"
    << "#include \"pc_eval_state.inc\"\n"
    << "  (void)pc;\n";
  for (size_t i = 0; i < n; ++i) {
    const XInsn &I = p.code[i];
    const size_t nx = i + 1 < n ? i + 1 : i;
    auto lbl = [&](size_t t) { return "L" + std::to_string(t < n ? t : n - 1); };
    o << lbl(i) << ": {\n"
      << "#define NEXT { goto " << lbl(nx) << "; }\n"
      << "#define JUMP_Z { goto " << lbl(I.c) << "; }\n"
      << "#define JUMP_W { goto " << lbl(I.e) << "; }\n"
      << "#define JUMP_2 { goto " << lbl(i + 2) << "; }\n"
      << "#define NEXT_INSN " << (i + 1 < n ? insn_literal(p.code[i + 1]) : insn_literal(I)) << "\n"
      << "  const uint4 I = " << insn_literal(I) << ";\n"
      << "  {\n" << case_text(I.opa & 0xffu) << "  }\n"
      << "#undef NEXT\n#undef JUMP_Z\n#undef JUMP_W\n#undef JUMP_2\n#undef NEXT_INSN\n"
      << "}\n";
  }
  o << "  return tos;\n"
    << "#undef PUSH\n#undef STK\n#undef BINF\n#undef BINI\n#undef IMM\n"
    << "}\n"
    << "}  // namespace\n"
    << "}  // namespace pc\n";
  o << "extern \"C\" __global__ void __launch_bounds__(" << kBlock << ") pc_jit_price(const pc::PriceArgs a) {\n"
    << "  pc::price_tiles<pc::D, " << (write ? "true" : "false") << ">(a, [&](const uint4 *P, const float *pool,\n"
    << "      float2 *R, const pc::Rng2 &g, bool live0, bool live1, const float (&Bm)[pc::D * pc::D],\n"
    << "      const float (&S0)[pc::D]) { return pc::jit_eval(P, pool, R, a, g, live0, live1, Bm, S0); });\n"
    << "}\n";
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
pc_status to_cubin(const Program &p, int d, bool write, const std::string &arch, std::vector<char> &cubin) {
  const std::string src = generate(p, d, write);
  nvrtcProgram prog = nullptr;
  nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "pc_jit.cu", kJitHeaderCount, kJitHeaderSrcs,
                                     kJitHeaderNames);
  if (r != NVRTC_SUCCESS) return nvrtc_fail(r, nullptr, "run-time compiler");
  const std::string a = "-arch=" + arch;
  const char *opts[] = {a.c_str(), "-std=c++17", "-default-device", "-DPC_JIT"};
  r = nvrtcCompileProgram(prog, 4, opts);
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

pc_status compile(const Program &p, int d, bool write, int device, cudaLibrary_t &lib, cudaKernel_t &kern) {
  cudaDeviceProp prop{};
  CU(cudaGetDeviceProperties(&prop, device), "device properties");
  std::vector<char> cubin;
  pc_status s = to_cubin(p, d, write, "sm_" + std::to_string(prop.major) + std::to_string(prop.minor) + "a",
                         cubin);
  if (s != PC_OK) return s;
  CU(cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0), "module load");
  cudaError_t e = cudaLibraryGetKernel(&kern, lib, "pc_jit_price");
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

pc_status jit_kernel(const pc_contract *k, int d, bool write, cudaKernel_t &out) {
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
    if (E.d == d && E.write == write && E.program == words) {
      out = E.kernel;
      return PC_OK;
    }
  }
  JitEntry E;
  E.program = words;
  E.d = d;
  E.write = write;
  pc_status s = compile(k->prog, d, write, c->device, E.lib, E.kernel);
  if (s != PC_OK) return s;
  out = E.kernel;
  c->jit_cache.emplace(h, std::move(E));
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
                                          int32_t p1, int32_t p2, int32_t d, size_t *cubin_bytes) {
  if (!cubin_bytes) return fail(PC_EINVAL, "null output");
  if (d < 1 || d > PC_MAX_UNDERLYINGS) return fail(PC_EINVAL, "d must be 1..4");
  Program p;
  std::string err;
  pc_status s = compile_program(bytecode, n_words, consts, n_consts, tparams, n_params, p1, p2, true, p, err);
  if (s != PC_OK) return fail(s, err);
  std::vector<char> cubin;
  s = to_cubin(p, d, false, "sm_103a", cubin);
  if (s != PC_OK) return s;
  *cubin_bytes = cubin.size();
  return PC_OK;
}
