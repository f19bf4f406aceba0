// pc_types.h -- device-visible structures of the pricing engine: the
// executable program, the model and layout images and the launch
// arguments.  Included by the kernels (nvcc) and by the run-time compiled
// kernels (NVRTC, which provides no C++ standard headers).
#pragma once

#ifdef __CUDACC_RTC__
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef unsigned long long uintptr_t;
#else
#include <cstddef>
#include <cstdint>
#endif

namespace pc {

// ---------------------------------------------------------------------------
// Executable program ("X-code"): what the loader emits and the kernel runs.
//
// The input bytecode is a postfix IL tree.  The loader rebuilds the tree,
// type-checks it, binds template variables (so every time expression becomes
// a static integer relative to the loopif offset t0), folds payoff to
// +-disc / 0, and emits a linear program for a warp-uniform stack machine:
// every lane of a warp executes the same instruction stream on its own path.
// if(c, a, b) becomes  c  IF  a  ELSE  b  SEL : IF/ELSE skip a branch that no
// live lane of the warp takes; SEL selects per lane.  loopif(c, a, b, n)
// becomes  LOOP  c  LTEST  a  LLATCH  LNEXT  b  LEND : the warp iterates
// k = 0..n with t0 = t0_entry + k, each lane latching the then-value at its
// first k whose test holds (Fig. 3), and leaves early once every live lane
// has latched.  Values are 32-bit: float for reals, int32 for nats and bools.
// ---------------------------------------------------------------------------
struct XInsn {
  uint32_t opa;  // opcode (low 8 bits) | A (24 bits)
  uint32_t b;
  uint32_t c;
  uint32_t e;
};
static_assert(sizeof(XInsn) == 16, "XInsn is one 16-byte shared-memory load");

enum XOp : uint32_t {
  X_END = 0,
  X_CONST,      // push bits b
  X_MODEL,      // A = label; push S_label(ordinal b + t0 - t_now)
  X_PAYOFF,     // A = 1 for negative sign; push +-c * disc(ordinal b + t0 - t_now), c float bits
  X_TIME,       // push int b + t0
  X_NOW,        // push int t_now
  X_NEGF, X_NOT,
  X_ADDF, X_SUBF, X_MULF, X_DIVF, X_MAXF, X_MINF, X_LTF, X_LEF, X_EQF,
  X_ADDI, X_SUBI, X_MULI, X_MAXI, X_MINI, X_LTI, X_LEI, X_EQI,
  X_AND, X_OR,
  // real op with an immediate right operand (float bits in b):  x op k
  X_ADDFK, X_SUBFK, X_MULFK, X_DIVFK, X_MAXFK, X_MINFK, X_LTFK, X_LEFK, X_EQFK,
  // immediate on the left:  k op x
  X_RSUBFK, X_RDIVFK, X_RLTFK, X_RLEFK,
  // X_MODEL followed by a real op with immediate c: S op k
  X_MODEL_MULK, X_MODEL_DIVK,
  X_IF,         // c = pc of the else branch; peek cond
  X_ELSE,       // c = pc of SEL
  X_SEL,        // pop else, then, cond -> push cond ? then : else
  X_LOOP,       // A = frame slot; b = bound n; c = pc of the loop's LTEST or LSTEPK
  X_LTEST,      // A = frame slot; c = pc of LNEXT
  X_LLATCH,     // A = frame slot
  X_LNEXT,      // A = frame slot; b = bound n; c = pc of loop condition; e = pc after LEND
  X_LEND,       // A = frame slot
  // Fused multi-asset ops (all leaves read at one static time b):
  // X_LRED: v = leaf_0 (op) leaf_1 (op) ... left to right, op = min / max /
  //   add; leaf_i = S_{l_i} [* or / pool[c + i]]; optionally compared with
  //   the immediate e.  A: bits 0-1 op (0 min, 1 max, 2 add), 2-3 scale
  //   (0 none, 1 mult, 2 div), 4-6 compare (0 none, 1 v<k, 2 v<=k, 3 k<v,
  //   4 k<=v), 8-9 leaves-1, 10-17 labels (2 bits each).
  X_LRED,
  // X_LANY: p = cmp(leaf_0, k) or/and cmp(leaf_1, k) ...  A: bit 0 combine
  //   (0 or, 1 and), 2-3 scale, 4-6 compare (1..4 as X_LRED), 8-9 leaves-1,
  //   10-17 labels; c = pool offset of the scales; e = immediate k.
  X_LANY,
  // X_LSTEPK: one loopif iteration whose then-branch is the literal
  //   pool[A >> 8]: pop the condition, latch the literal on newly true lanes,
  //   then continue as X_LNEXT.  A: bits 0-7 frame slot, 8-23 pool index;
  //   b = bound n; c = pc of the loop condition; e = pc after X_LEND.
  X_LSTEPK,
  // X_LOOPANY: a whole loopif whose condition is one X_LRED-with-compare or
  //   X_LANY instruction (stored right after, as a descriptor that is not
  //   dispatched) and whose then-branch is the literal pool[A >> 8]: tests
  //   k = 0..n in a device loop, latching the literal; when every live lane
  //   latched, pushes the results and jumps to e (after X_LEND); otherwise
  //   fills the frame (A & 0xff) and runs the else-branch at pc + 2, which
  //   X_LEND closes.  b = bound n.
  X_LOOPANY,
  X_NUM_OPS
};

// Loop frame layout on the operand stack (slot offsets from the frame base).
enum { LF_K = 0, LF_T0 = 1, LF_DONE = 2, LF_RES = 3, LF_NEWLY = 4, LF_SLOTS = 5 };

// ---------------------------------------------------------------------------
// Brownian-bridge schedule in date order (device).
//
// Dates are produced lazily in time order.  The bridge keeps W of the last
// produced date in registers and a stack of already-computed W of later
// dates.  To produce date t the kernel runs the ops of t: each computes
// bridge node m from (W_cur, W_top) and pushes it, except the last op, whose
// result is W_t itself; a date with no ops pops W_t from the stack.
//
// Normals: the ops are numbered k = 0, 1, ... in the order the walk runs
// them (every path runs the same sequence), and op k takes the d normals
// m = d k + i (underlying i < d) of the path: Philox counter m >> 2, word
// m & 3.  So the normals are used in counter order, four per Philox block,
// none left over; a node whose normals start inside the block of the
// previous node takes them from the registers that kept that block's later
// words (for d < 4 at most three).
// ---------------------------------------------------------------------------
struct BridgeOp {
  float wl, wl_, wr, wr_;  // endpoint weights, each twice: a packed pair for the lane's two paths
  float sd, sd_;           // conditional standard deviation, twice
  uint32_t j;              // breadth-first node number (diagnostics)
  uint16_t flags;          // BR_* below
  uint16_t m;              // date ordinal produced (diagnostics)
};
static_assert(sizeof(BridgeOp) == 32, "BridgeOp layout: two 16-byte loads");

enum : uint16_t {
  BR_ROOT = 1,  // first node (last date): W = sd * z (its wl = wr = 0)
};

// Device image of a model (one allocation, offsets in bytes).
struct ModelDev {
  const int32_t *date_ops;  // [n+2] op range of date t: [date_ops[t], date_ops[t+1])
  const BridgeOp *ops;      // [n]
  const float2 *A;          // [(n+1)*d] log2(e)(r - sigma^2/2) tau_o (S = S0 2^(A + B W)), each twice
  const float *B;           // [d*d]     log2(e) sigma_i L_ik
  const float *disc;        // [n_hist+n+1] disc of ordinal o at index o + n_hist
  const float *sval;        // [(n_hist+1)*d] value of label l at ordinal o <= 0, index (o+n_hist)*d+l
  // pathwise tangents (greeks)
  const float *tau;         // [n+1] year fraction of ordinal o
  const float *L;           // [d*d] Cholesky factor (row-major)
  const float *sig;         // [d] volatilities
  int32_t d, n, n_hist, t_now;
  int32_t n_levels;         // bisection levels
  int32_t bstack;           // bridge stack depth
  // B and S0 by value: in a kernel parameter they are read from the
  // constant bank where used, and take no registers
  float Bv[16];             // B row-major over d x d (the first d*d entries)
  float S0v[4];             // S0 of each underlying
};

// Per-thread shared-memory region: 32-bit words, word w of thread t at
// region[w * BLOCK + t] (uniform w -> conflict-free).
struct Layout {
  int32_t stack;      // operand stack words
  int32_t off_bstack; // bridge stack (bstack * d)
  int32_t off_cache;  // = off_win (no shared-memory caches)
  int32_t off_win;    // date window (win * d)
  int32_t off_xwin;   // window of X = L W (win * d), sensitivity kernel only
  int32_t words;      // total words per thread in shared memory
  int32_t win;        // window size (power of two)
  // HBM window (programs whose lookback does not fit shared memory): the
  // window of thread t of the launch is column t of gwin, slot s at
  // gwin[s * gstride + t] (gstride = grid * block); null for the shared window.
  float2 *gwin;
  int64_t gstride;
};

constexpr int kBlock = 128;          // largest block of the pricing kernel (32..128 threads)
constexpr int kPathsPerLane = 2;     // paths a lane carries at once (float2 values)
constexpr int kTilePaths = 32 * kPathsPerLane;

// Dynamic shared memory of the pricing kernel: program (16 B per
// instruction), constant pool (padded to 4 floats), and the per-thread
// region of float2 slots.
inline size_t price_smem_bytes(size_t n_insn, size_t n_pool_padded, int words, int block) {
  return n_insn * 16 + n_pool_padded * 4 + size_t(words) * block * 8;
}

struct RoundKeys {
  uint32_t k[20];
};

// Philox4x32-10 round keys of a 64-bit seed: round r XORs (key0 + r W0,
// key1 + r W1), the key bumped by the Weyl constants between rounds.
inline void philox_round_keys(uint64_t seed, uint32_t *rk) {
  uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = k0;
    rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

struct PriceArgs {
  const XInsn *prog;        // program followed by its constant pool
  int32_t n_insn;
  int32_t n_pool;           // pool floats, padded to a multiple of 4
  ModelDev m;
  Layout lay;
  uint64_t n_paths, path_offset;
  uint32_t key0, key1, stream;
  uint32_t rk[20];          // Philox round keys: (key0 + r W0, key1 + r W1) for r = 0..9
  uint64_t n_tiles;
  int32_t width;            // doubles per tile partial (2 for prices)
  uint32_t chunk_tiles;     // tiles per reduction chunk
  uint32_t n_chunks;        // ceil(n_tiles / chunk_tiles) <= kMaxChunks
  double *tile_partials;    // [n_tiles * width] scratch
  unsigned char *control;   // kControlBytes of scratch, zero between launches (see below)
  double *out;              // [width + 1]: sums over all paths, then n_paths
  float *out_paths;         // nullable: per-path payoffs (sensitivities: 3 floats per path)
  int32_t *status;          // device status word (nonzero = error)
  int32_t greek_label;      // sensitivity kernel: the underlying g of the tangents
};

// The adjoint sensitivity kernel's tape (pc_adjoint.cuh): one region per
// resident warp of the launch, entry e of lane l at [e * 32 + l].
struct TapeArgs {
  float4 *part;   // [warp][emax][32]: (p1 of both paths, p2 of both paths)
  float2 *adj;    // [warp][emax][32]: adjoints of both paths
  int2 *ids;      // [warp][emax]: input entries (in1, in2); a leaf: in1 = -2 - label
  int32_t emax;   // entries per warp region
};

// Reduction scratch "control" block (zero between launches; every launch
// leaves it zero): 64-bit counters at byte 0 (next tile, finished blocks,
// finished chunks), 32-bit per-chunk tile counters at kChunkCountOff, and
// the chunk partials (width doubles each) at kChunkPartOff.
constexpr int kMaxChunks = 256;
constexpr size_t kChunkCountOff = 256;
constexpr size_t kChunkPartOff = 2048;
constexpr size_t kControlBytes = kChunkPartOff + size_t(kMaxChunks) * 8 * sizeof(double);
inline void reduction_chunks(uint64_t n_tiles, uint32_t &chunk_tiles, uint32_t &n_chunks) {
  uint64_t c = (n_tiles + kMaxChunks - 1) / kMaxChunks;
  if (c < 64) c = 64;
  chunk_tiles = uint32_t(c);
  n_chunks = uint32_t((n_tiles + c - 1) / c);
}

}  // namespace pc
