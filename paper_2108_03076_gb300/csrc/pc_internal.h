// pc_internal.h -- structures shared by the host side (loader, model setup,
// C ABI) and the device kernels of the pricing engine.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "pc.h"
#include "pc_types.h"

namespace pc {
// Kernel launchers (pc_kernels.cu).  All return a cudaError_t.
cudaError_t launch_price(const PriceArgs &a, int grid, int block, size_t smem_bytes, cudaStream_t s);
cudaError_t launch_greeks(const PriceArgs &a, int grid, int block, size_t smem_bytes, cudaStream_t s);
int greeks_blocks_per_sm(int d, int block, size_t smem_bytes);
cudaError_t launch_debug_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                size_t n, cudaStream_t s);
cudaError_t launch_debug_paths(const ModelDev &m, const Layout &lay, uint64_t n_paths,
                               uint64_t offset, uint32_t k0, uint32_t k1, uint32_t stream,
                               float *out, cudaStream_t s);
int price_blocks_per_sm(int d, int block, size_t smem_bytes, bool hbm_window, bool memoise = true);

// Portfolio pricing (one persistent launch per group of contracts with the
// same underlying count and a similar per-path footprint).  A work unit is a
// run of consecutive tiles of one contract; warps take units from the
// group's counter in the order of the unit array (costliest first) and run
// their tiles exactly as the single-contract kernel does, finishing each
// tile into that contract's own reduction scratch.
struct BatchUnit {
  uint32_t item;     // index into the per-contract argument array
  uint32_t n_tiles;  // tiles in the unit (>= 1)
  uint64_t tile0;    // first tile
};
static_assert(sizeof(BatchUnit) == 16, "BatchUnit is 16 bytes");
struct BatchArgs {
  const PriceArgs *items;       // per-contract arguments (device)
  const BatchUnit *units;       // this group's units (device)
  uint32_t n_units;
  uint32_t slot_bytes;          // per-warp slot: arguments + program + pool
  unsigned long long *counter;  // next unit; zero before the launch
};
// Per-warp slot in shared memory (a contract's arguments, then its program
// and constant pool), ahead of the per-thread regions.
constexpr size_t kBatchArgsBytes = (sizeof(PriceArgs) + 15) & ~size_t(15);
// A warp's slot holds its unit's arguments; programs and pools are read
// from global memory through L1 (a slot sized for the group's largest
// program -- up to 6.5 KB -- cost half the resident warps).
inline size_t batch_slot_bytes(size_t n_insn, size_t n_pool_padded) {
  (void)n_insn;
  (void)n_pool_padded;
  return kBatchArgsBytes;
}
inline size_t batch_smem_bytes(size_t slot_bytes, int words, int block) {
  return slot_bytes * size_t(block / 32) + size_t(words) * size_t(block) * sizeof(float) * kPathsPerLane;
}
// Sets the kernel's dynamic shared-memory limit and returns its resident
// blocks per SM (0 if it cannot run).  Call before any stream capture.
int batch_blocks_per_sm(int d, int block, size_t smem_bytes);
cudaError_t launch_batch(const BatchArgs &b, int d, int grid, int block, size_t smem_bytes,
                         cudaStream_t s);
// The adjoint sensitivity kernel (pc_adjoint.cuh): launch, and resident
// blocks per SM for a shared-memory footprint (sets the kernel's limit).
cudaError_t launch_adjoint(const PriceArgs &a, const TapeArgs &t, int grid, int block, size_t smem,
                           cudaStream_t s);
int adjoint_blocks_per_sm(int d, int block, size_t smem_bytes);
// Occupancy results keyed by (device, kernel variant, block, shared memory):
// the query runs once per key (it sets the kernel's shared-memory limit and
// costs microseconds), later calls return the stored count.  With `store`
// false a missing key is queried and not stored (no host allocation).
int occupancy_memo(uint64_t variant, int block, size_t smem, int (*query)(uint64_t, int, size_t),
                   bool store = true);

// Device address and size of the fixed scratch array used by
// pc_price_noalloc on the current device (looked up once per device).
cudaError_t noalloc_scratch(void **ptr, size_t *bytes);
constexpr size_t kNoAllocCounterBytes = kControlBytes;
int max_dynamic_smem();

// ---------------------------------------------------------------------------
// Host-side program handling (pc_program.cpp)
// ---------------------------------------------------------------------------
struct Program {
  std::vector<XInsn> code;
  std::vector<float> pool;  // constants of fused ops (scales, loop literals)
  pc_program_info info{};
  int32_t frame_slots = 0;  // stack slots (values + frames)
};

// Decode, verify, bind and compile bytecode.  On failure returns a PC_E*
// code and sets `err`.
pc_status compile_program(const uint32_t *words, size_t n_words, const double *consts,
                          size_t n_consts, const int32_t *tparams, size_t n_params,
                          int32_t p1, int32_t p2, bool bind_parties, Program &out,
                          std::string &err);

// Abstract run of the executable form with every branch taken, as the warp
// would run it if some lane took each branch at every loop iteration: gives
// every ordinal the program can touch and the largest lookback below the
// frontier of generated dates.  Skipping branches only lowers the frontier
// at any later point, so this bound holds for every actual run.  No heap
// use: pc_price_noalloc runs it too.  On the first failure it stops and
// calls on_fail(status, time, ordinal) (time and ordinal of an out-of-grid
// read; 0 for PC_ELIMIT, a program whose loop trip counts exceed 2^26
// analysis steps).
//
// The walk also counts `entries`: an upper bound on the entries a run of
// the program appends to the adjoint tape (pc_adjoint.cuh): one per model
// read, real arithmetic operation, select, loop latch and loop end, and
// 2n - 1 per fused n-leaf reduction (none for tests).
template <typename OnFail>
struct TimeWalk {
  const XInsn *C;
  int64_t t_now, n_dates, n_hist;
  OnFail on_fail;
  int64_t frontier = 0, lookback = 0, steps = 0, entries = 0;
  pc_status st = PC_OK;

  static int64_t entry_count(const XInsn &I) {
    const uint32_t op = I.opa & 0xffu;
    switch (op) {
      case X_MODEL: case X_MODEL_MULK: case X_MODEL_DIVK:
      case X_NEGF: case X_ADDF: case X_SUBF: case X_MULF: case X_DIVF: case X_MAXF: case X_MINF:
      case X_ADDFK: case X_SUBFK: case X_MULFK: case X_DIVFK: case X_MAXFK: case X_MINFK:
      case X_RSUBFK: case X_RDIVFK: case X_SEL:
        return 1;
      case X_LRED: {
        const uint32_t A = I.opa >> 8;
        return ((A >> 4) & 7u) ? 0 : 2 * int64_t(((A >> 8) & 3u) + 1) - 1;
      }
      default:
        return 0;
    }
  }

  void run(size_t a, size_t b, int64_t t0) {
    for (size_t pc = a; pc < b && st == PC_OK;) {
      if (++steps > (int64_t(1) << 26)) {
        st = PC_ELIMIT;
        on_fail(st, 0, 0);
        return;
      }
      const XInsn &I = C[pc];
      const uint32_t op = I.opa & 0xffu;
      if (op == X_MODEL || op == X_MODEL_MULK || op == X_MODEL_DIVK || op == X_PAYOFF ||
          op == X_LRED || op == X_LANY) {
        const int64_t o = int64_t(int32_t(I.b)) + t0 - t_now;
        if (o < -n_hist || o > n_dates) {
          st = PC_ERANGE;
          on_fail(st, int64_t(int32_t(I.b)) + t0, o);
          return;
        }
        if (op != X_PAYOFF && o > 0) {
          if (o > frontier) frontier = o;
          else if (frontier - o > lookback) lookback = frontier - o;
        }
        entries += entry_count(I);
        ++pc;
      } else if (op == X_LOOPANY) {
        const int64_t n = I.b;
        const size_t end = I.e;  // pc after LEND
        for (int64_t k = 0; k <= n && st == PC_OK; ++k) run(pc + 1, pc + 2, t0 + k);
        run(pc + 2, end - 1, t0 + n);
        entries += 1;  // LEND
        pc = end;
      } else if (op == X_LOOP) {
        const int64_t n = I.b;
        const size_t cond = pc + 1, test = I.c;
        if ((C[test].opa & 0xffu) == X_LSTEPK) {
          const size_t end = C[test].e;  // pc after LEND
          for (int64_t k = 0; k <= n && st == PC_OK; ++k) run(cond, test, t0 + k);
          run(test + 1, end - 1, t0 + n);  // else-branch (before LEND)
          entries += (n + 1) + 1;          // LSTEPK per iteration, LEND
          pc = end;
          continue;
        }
        const size_t next = C[test].c;
        const size_t end = C[next].e;  // pc after LEND
        for (int64_t k = 0; k <= n && st == PC_OK; ++k) {
          run(cond, test, t0 + k);
          run(test + 1, next - 1, t0 + k);  // then-branch (before LLATCH)
        }
        run(next + 1, end - 1, t0 + n);  // else-branch (before LEND)
        entries += (n + 1) + 1;          // LLATCH per iteration, LEND
        pc = end;
      } else if (op == X_END) {
        return;
      } else {
        entries += entry_count(I);
        ++pc;
      }
    }
  }

  // the window (power of two) that holds the largest lookback
  int32_t window() const {
    int32_t w = 1;
    while (w < lookback + 1) w <<= 1;
    return w;
  }
};

// Static analysis of a program against a model's time layout (TimeWalk):
// every model and payoff time within [-n_hist, n] as ordinals; `win`
// receives the window size needed (power of two, <= 2 * PC_MAX_DATES:
// callers decide where such a window can live).
pc_status analyse_program(const Program &p, int32_t t_now, int32_t n_dates, int32_t n_hist,
                          int32_t &win, std::string &err);

// cutPayoff (Sec. 4.1) on bytecode: every payoff(t, p1', p2') becomes
// if(t < now, 0, payoff(t, p1', p2')); the literal 0.0 is appended to the
// constants unless present.
pc_status cut_payoff(const uint32_t *words, size_t n_words, const double *consts, size_t n_consts,
                     std::vector<uint32_t> &out, std::vector<double> &out_consts, std::string &err);

pc_status assemble_text(const char *text, std::vector<uint32_t> &words,
                        std::vector<double> &consts, std::string &err);

// ---------------------------------------------------------------------------
// Host-side model setup (pc_model.cpp)
// ---------------------------------------------------------------------------
struct ModelHost {
  int32_t d = 0, n = 0, n_hist = 0, t_now = 0;
  std::vector<double> S0, sigma, corr, L;  // L: Cholesky factor, row-major
  double r = 0;
  std::vector<int32_t> day, hist_day;
  std::vector<double> history;
  // device tables, host copies
  std::vector<int32_t> date_ops;
  std::vector<BridgeOp> ops;
  std::vector<float2> A;  // drift exponents, each twice (packed pairs)
  std::vector<float> B, disc, sval, tau, Lf, sig;
  int32_t n_levels = 0, bstack = 0;
};

pc_status build_model(const pc_model_desc &desc, ModelHost &out, std::string &err);

}  // namespace pc
