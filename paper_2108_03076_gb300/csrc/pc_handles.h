// pc_handles.h -- the opaque handles of include/pc.h and the host helpers
// shared by the entry-point files (pc_capi.cpp, pc_batch.cpp).  Private to
// the library.
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "pc.h"
#include "pc_internal.h"

// A run-time specialised pricing kernel: the program it was compiled from
// (code and pool words), the underlying count and the per-path variant.
// Kinds of run-time specialised kernels: pricing (bit kJitPriceWrite: with
// per-path payoffs; bit kJitHbm: the window of dates in HBM; bit
// kJitWinRegs: a window of one date, kept in registers; bit kJitPairs2 (with
// kJitWinRegs): four paths a lane), and the
// control-variate kernel (kJitCv + its kCv* mode bits), the tangent kernel
// (kJitGreeks, + 1: per-path outputs) and the adjoint kernel (kJitAdjoint,
// + 1: per-path outputs).
constexpr int kJitPrice = 0, kJitPriceWrite = 1, kJitHbm = 2, kJitWinRegs = 4, kJitPairs2 = 8, kJitCv = 16,
              kJitGreeks = 32, kJitAdjoint = 64;
// resident blocks per SM the specialised pricing kernel's register bound is
// set for by default (<= 72 registers at 128 threads: the fastest measured)
constexpr int kJitMinBlocks = 7;
// resident blocks per SM the specialised control-variate kernel's register bound is set for
constexpr int kJitCvMinBlocks = 5;
// dates of the model from which a one-date-window kernel takes two path pairs a lane
constexpr int kJitPairsMinDates = 64;
constexpr size_t kJitStaticSmem = 256;  // bound on price_tiles' static shared memory

struct JitEntry {
  std::vector<uint32_t> program;
  int d = 0;
  int kind = kJitPrice;
  int block = 0;  // the launch block the kernel is compiled for (its slot stride)
  int min_blocks = 0;  // its launch bound's resident blocks per SM (0: the kernel's own)
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
};

struct pc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  int max_smem = 0;
  int sm_smem = 0;       // shared memory per SM (bytes)
  int smem_reserve = 0;  // shared memory the system reserves per resident block (bytes)
  double *d_res = nullptr;       // [8]: sum, sumsq, n, -, status word (int32 at d_res+4)
  double *d_gout = nullptr;      // [PC_MAX_UNDERLYINGS * 8]: sensitivity sums per underlying
  double *d_partials = nullptr;  // tile partials (scratch)
  size_t partial_cap = 0;        // doubles
  unsigned char *d_control = nullptr;  // reduction control block (kControlBytes, zero between launches)
  void *d_tape = nullptr;        // adjoint tapes, one region per resident warp (grow-only)
  size_t tape_cap = 0;           // bytes
  float2 *d_gwin = nullptr;      // HBM windows of simulated dates (grow-only)
  size_t gwin_cap = 0;           // float2 slots
  int32_t window_mode = 0;       // PC_WINDOW_AUTO / _SHARED / _HBM
  int32_t jit = 0;               // 1: price with run-time specialised kernels
  // streams and events of one-shot portfolio launches (pc_price_batch),
  // created once per context
  std::vector<cudaStream_t> batch_aux;
  std::vector<cudaEvent_t> batch_join;
  cudaEvent_t batch_fork = nullptr;
  int32_t cv_min_blocks = 0;     // launch bound of the specialised control-variate kernel (0: its default)
  int32_t jit_pairs = 0;         // path pairs a lane of a specialised kernel with a one-date window (0 automatic, 1 or 2)
  std::mutex jit_mu;
  std::multimap<uint64_t, JitEntry> jit_cache;  // program hash -> compiled kernels
  std::map<std::pair<const void *, size_t>, int> jit_occ;  // (kernel, smem) -> resident blocks
  cudaMemPool_t pool = nullptr;  // stream-ordered allocations of contracts (null: cudaMalloc)
  double *h_res = nullptr;       // pinned [16]: results read back by the blocking calls
  // pinned staging of program uploads, two halves filled in turn: a half is
  // reused once the event recorded when it was left has completed
  uint32_t *h_stage = nullptr;
  size_t stage_words = 0;        // words per half
  size_t stage_off = 0;          // next free word in the current half
  int stage_half = 0;
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  bool stage_pending[2] = {false, false};
  // compiled programs by their inputs (bytecode, constants, template
  // parameters, parties): reloading a program skips the compiler
  std::mutex load_mu;
  std::multimap<uint64_t, std::pair<std::vector<uint32_t>, pc::Program>> program_cache;
  double timeout_s = 300.0;
  int32_t fail_allocs = 0;       // failure injection: this many next allocations fail (pc_debug_fail_allocations)
  int live_objects = 0;
};

struct pc_model {
  pc_ctx *ctx = nullptr;
  pc::ModelHost H;
  void *d_mem = nullptr;
  pc::ModelDev dev{};
  uint64_t id = 0;
};


struct pc_contract {
  pc_ctx *ctx = nullptr;
  pc::Program prog;
  pc::XInsn *d_code = nullptr;
  bool pooled = false;            // d_code came from the context's memory pool
  std::vector<uint32_t> image;    // program then padded pool: the uploaded words
  std::mutex mu;
  std::map<std::pair<uint64_t, uint64_t>, int32_t> win_cache;  // (model id, layout key) -> window
};

namespace pc {

// Device memory on the context's stream: from its memory pool (stream
// ordered, no device synchronisation) when it has one, else cudaMalloc.
cudaError_t ctx_alloc(pc_ctx *c, void **p, size_t bytes, bool &pooled);
void ctx_free(pc_ctx *c, void *p, bool pooled);
// Resident blocks per SM of a run-time compiled kernel at this dynamic
// shared memory (sets its shared-memory limit on first use; memoised).
cudaError_t jit_occupancy(pc_ctx *c, const void *kern, int block, size_t smem, int &blocks);

// Record a message for pc_last_error and return the status.
pc_status fail(pc_status s, const std::string &m);
pc_status cuda_fail(cudaError_t e, const char *what);

#define CU(call, what)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return ::pc::cuda_fail(e_, what); \
  } while (0)

// Wait for the context's stream with its wall-clock limit.
pc_status wait_stream(pc_ctx *c);

// cudaMalloc for the context's buffers, or a simulated out-of-memory
// (cudaErrorMemoryAllocation, nothing allocated) while the context's
// failure injection count is positive.
cudaError_t ctx_malloc(pc_ctx *c, void **p, size_t bytes);

// Room left for a kernel's static shared memory when sizing its dynamic
// shared memory.
constexpr size_t kStaticSmemReserve = 2048;

// Constant-pool floats of a program, rounded up to whole 16-byte words.
size_t pool_padded(const Program &p);

// A pricing launch: per-contract arguments plus its single-launch shape.
struct Launch {
  PriceArgs args{};
  int grid = 0;
  int block = kBlock;
  size_t smem = 0;
  bool hbm_window = false;  // window in HBM (args.lay.gwin set by the launcher)
};

// Validate (model, contract, n_paths), resolve the contract's date window for
// the model and fill the per-contract arguments (everything but the
// reduction scratch and outputs) and a single-launch shape.  With
// allow_hbm the window may be placed in HBM (pricing kernel only): when the
// context asks for it, or (automatic mode) when the shared window would
// leave fewer than 8 resident warps per SM or exceeds PC_MAX_WINDOW.
pc_status prepare(const pc_model *m, const pc_contract *k, uint64_t n_paths, uint64_t offset,
                  uint64_t seed, uint32_t stream, Launch &L, bool allow_hbm = false);

// Grow the context's tile-partial scratch to at least `doubles`.
pc_status ensure_partials(pc_ctx *c, size_t doubles);

// The run-time specialised kernel of the contract's program for d
// underlyings, a kernel kind (kJit*) and the launch's block size (the
// per-thread slot stride, a constant in the compiled code); compiled on
// first use, cached on the context by program content.
// min_blocks: for pc_jit_price, the resident blocks per SM its launch bound
// asks for (0: the default, 7); other kinds fix their own bound.
pc_status jit_kernel(const pc_contract *k, int d, int kind, int block, cudaKernel_t &out, int min_blocks = 0);
// Programs of at most PC_JIT_MAX_INSNS instructions are specialised; the
// launches of longer ones interpret them.
bool jit_eligible(const pc_contract *k);
// A program the specialised adjoint kernel takes (its date generator is
// inlined at each reading instruction: a few of them at most).
bool adjoint_jit_eligible(const pc_contract *k);
// Compile the specialised kernels of many requests into the context's cache
// (those not there yet), NVRTC on the host's cores in parallel; jit_kernel
// then finds them.
struct JitRequest {
  const pc_contract *k;
  int d, kind, block, min_blocks;
};
pc_status jit_compile_many(pc_ctx *c, const std::vector<JitRequest> &reqs);
// The specialised pricing kernel's variant for a prepared launch (window in
// registers, path pairs a lane, HBM window), its layout (the launch's shared
// memory; may re-choose the block) and the register bound it is compiled for.
int jit_window_kind(const pc_ctx *c, const Launch &L);
size_t jit_layout(const pc_ctx *c, const pc_contract *k, Launch &L, int bits);
int jit_min_blocks(const pc_ctx *c, size_t smem, int block);
void jit_release(pc_ctx *c);

// Turn a raised device status word into PC_EDEVICE (and clear it).
pc_status check_status(pc_ctx *c, int32_t status);

}  // namespace pc
