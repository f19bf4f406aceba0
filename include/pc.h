/*
 * pc.h -- C ABI of the payoff-expression Monte Carlo pricing engine (sm_103a).
 *
 * The engine prices contracts that were compiled into the payoff intermediate
 * language (IL) of Annenkov & Elsman, "Certified Compilation of Financial
 * Contracts" (PPDP'18): the expression language of Sec. 3 (now, model(l, t),
 * if, loopif, payoff(t, p1, p2), unary and binary operators, literals,
 * template time expressions) with the semantics of Fig. 3.  A contract arrives
 * as postfix bytecode plus the values of its template variables (the
 * "instrument" of Sec. 2 instantiated without recompiling, Sec. 6.2); it is
 * valued by Monte Carlo over a correlated Black-Scholes market whose paths
 * play the role of the external environment rho of Fig. 3.
 *
 * Conventions for every entry point:
 *   - Every function returns a pc_status; PC_OK (0) on success, a negative
 *     code on failure.  Nothing aborts, throws or exits across this ABI.
 *     A failed call leaves its outputs untouched and sets a message that
 *     pc_last_error() returns.
 *   - Host arrays passed in are read during the call and copied as needed;
 *     the caller keeps ownership.  Handles are opaque and owned by the
 *     library until their *_destroy call.
 *   - Pointers documented as "device" must point to memory of the context's
 *     device; all other pointers are host pointers.
 *   - All work of a context runs in order on the context's CUDA stream.
 *   - Thread safety: calls on different contexts may run concurrently; calls
 *     on one context must be serialised by the caller.
 */
#ifndef PC_H
#define PC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pc_status;

#define PC_OK          0
#define PC_EINVAL     -1   /* bad argument (null pointer, size out of range)        */
#define PC_EBYTECODE  -2   /* malformed program: bad opcode or operand, stack        */
                           /* underflow, leftover values, type mismatch              */
#define PC_ETPARAM    -3   /* template variable unbound or negative                  */
#define PC_ERANGE     -4   /* a model/payoff time falls outside the model's grid or  */
                           /* history, or the lookback exceeds the engine's window  */
#define PC_ENOTPD     -5   /* correlation matrix not symmetric positive definite    */
#define PC_ENOMEM     -6   /* host or device allocation failed                       */
#define PC_ECUDA      -7   /* a CUDA runtime call failed                              */
#define PC_ETIMEOUT   -8   /* the device did not finish within the context's limit   */
#define PC_EDEVICE    -9   /* the kernel raised its device status word               */
#define PC_ELIMIT    -10   /* program or model exceeds a documented engine limit      */
#define PC_ESYNTAX   -11   /* pc_assemble: text is not valid IL                       */

/* Engine limits. */
#define PC_MAX_UNDERLYINGS   4      /* d                                            */
#define PC_MAX_DATES      8192      /* simulated dates per model                    */
#define PC_MAX_HISTORY    4096      /* history ordinals per model                   */
#define PC_MAX_PROGRAM   65536      /* bytecode words per program                   */
#define PC_MAX_CONSTS    16384      /* real literals per program                    */
#define PC_MAX_TPARAMS    1024      /* template variables per program               */
#define PC_MAX_STACK        96      /* operand stack depth (values + loop frames)   */
#define PC_MAX_WINDOW      256      /* lookback window kept in shared memory        */

/* ------------------------------------------------------------------------ */
/* Bytecode (input format of pc_load_payoff)                                 */
/* ------------------------------------------------------------------------ */
/*
 * A program is the postfix (children first, left to right) serialisation of
 * one IL expression tree (Sec. 3 grammar).  Each instruction is one header
 * word  op | (A << 8)  (op in the low 8 bits, A an unsigned 24-bit operand),
 * optionally followed by operand words:
 *
 *   PC_OP_REAL    A = index into consts[]          push real literal
 *   PC_OP_BOOL    A = 0 / 1                         push bool literal
 *   PC_OP_NAT     A = value                         push nat literal
 *   PC_OP_NOW                                       push t ("now", Fig. 3)
 *   PC_OP_TEXPR   + TIME(nat)                       push T[t]delta + t0
 *   PC_OP_MODEL   A = label, + TIME(int)            push rho(l, T[t]delta + t0)
 *   PC_OP_PAYOFF  + word p1' + word p2' + TIME(nat) push +-d(T[t]delta + t0) or 0
 *   PC_OP_NEG, PC_OP_NOT                            unary, pop 1 push 1
 *   PC_OP_ADD .. PC_OP_MIN                          binary, pop 2 push 1
 *   PC_OP_IF                                        pop cond, then, else
 *   PC_OP_LOOPIF  + TIME(bound)                     pop cond, then, else
 *
 * TIME is a sum of terms: one count word c (0..16) then c term words; a term
 * word with bit 31 set is template variable number (w & 0x7fffffff), else a
 * signed integer literal in bits 0..30 (two's complement of 31 bits).  This
 * is the flattened form of the tplus trees of ILTExpr / ILTExprZ (Sec. 5):
 * model times (ILTExprZ) may hold negative literals; texpr and payoff times
 * (ILTExpr) and the loopif bound (TExpr: one literal or one variable) must
 * be natural.
 *
 * Operand order for IF / LOOPIF is cond, then, else (pushed in that order).
 * Types follow Fig. 3: reals, bools and nats; arithmetic and comparisons
 * need operands of one type; nat subtraction truncates at 0; div is real.
 */
enum pc_opcode {
  PC_OP_REAL = 1, PC_OP_BOOL, PC_OP_NAT, PC_OP_NOW, PC_OP_TEXPR, PC_OP_MODEL,
  PC_OP_PAYOFF, PC_OP_NEG, PC_OP_NOT,
  PC_OP_ADD, PC_OP_SUB, PC_OP_MULT, PC_OP_DIV, PC_OP_LT, PC_OP_LE, PC_OP_EQ,
  PC_OP_AND, PC_OP_OR, PC_OP_MAX, PC_OP_MIN,
  PC_OP_IF, PC_OP_LOOPIF
};

/* ------------------------------------------------------------------------ */
/* Handles and descriptors                                                   */
/* ------------------------------------------------------------------------ */

typedef struct pc_ctx pc_ctx;
typedef struct pc_model pc_model;
typedef struct pc_contract pc_contract;

/*
 * Correlated Black-Scholes market on a date grid (the external environment
 * rho of Sec. 2 / Fig. 3 is one simulated path of this market).
 *
 * IL time t is grid ordinal o = t - t_now.  Ordinal 0 is the valuation date
 * (label l has value S0[l], discount 1); ordinals 1..n_dates are simulated
 * at calendar day day[o-1] (year fraction day/365); ordinals -1..-n_hist are
 * history: label l at ordinal -k is history[(k-1)*d + l], discounted with
 * day hist_day[k-1] (< 0).  Discount d(t) = exp(-r * day(o) / 365).
 * Paths: Brownian bridge over the grid, W -> X = L W with L the Cholesky
 * factor of corr, S_l(o) = S0[l] exp((r - sigma_l^2/2) tau_o + sigma_l X_l(o)).
 */
typedef struct pc_model_desc {
  int32_t d;                /* underlyings (labels 0..d-1), 1..PC_MAX_UNDERLYINGS */
  const double *S0;         /* [d] spot values, > 0                                */
  const double *sigma;      /* [d] volatilities, >= 0                              */
  const double *corr;       /* [d*d] row-major correlation, symmetric PD, diag 1   */
  double r;                 /* continuously compounded rate                        */
  int32_t n_dates;          /* simulated dates, 1..PC_MAX_DATES                    */
  const int32_t *day;       /* [n_dates] strictly increasing, > 0                  */
  int32_t t_now;            /* IL time of the valuation date (>= 0; "now")         */
  int32_t n_hist;           /* history ordinals, 0..PC_MAX_HISTORY                 */
  const double *history;    /* [n_hist*d] or NULL when n_hist == 0                 */
  const int32_t *hist_day;  /* [n_hist] < 0, strictly decreasing; NULL if none     */
} pc_model_desc;

/* Static facts about a verified program (pc_verify_payoff). */
typedef struct pc_program_info {
  int32_t n_nodes;          /* IL nodes                                            */
  int32_t n_insn;           /* instructions of the executable form                 */
  int32_t max_stack;        /* operand stack depth incl. loop frames               */
  int32_t result_is_real;   /* 1 when the expression is real-valued                */
  int32_t n_loops;          /* loopif nodes with a non-zero bound                  */
  int32_t n_tparams_used;   /* highest template variable index used + 1            */
} pc_program_info;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device` that issues all work on
 * `cuda_stream` (a cudaStream_t, borrowed, not destroyed by the library), or
 * on a stream the context creates when cuda_stream is NULL.  Allocates the
 * context's device scratch (reduction partials, status word).
 * Errors: PC_EINVAL, PC_ECUDA (no such device / not sm_103), PC_ENOMEM. */
pc_status pc_create(pc_ctx **out, int device, void *cuda_stream);

/* Wait for the context's work, free its device memory and the handle.
 * Models and contracts created on it must be destroyed first. */
pc_status pc_destroy(pc_ctx *ctx);

/* Message of the most recent failure on this thread (library-owned, valid
 * until the thread's next failing call); "" if none.  ctx may be NULL. */
/* Wall-clock limit of the context's blocking calls (seconds > 0; default
 * 300, or the environment variable PC_TIMEOUT_S at pc_create): a call whose
 * device work has not finished by then returns PC_ETIMEOUT.  The work is
 * not cancelled -- it completes on the context's stream, and later calls
 * are ordered after it, so the context stays usable.  Errors: PC_EINVAL. */
pc_status pc_set_timeout(pc_ctx *ctx, double seconds);

const char *pc_last_error(const pc_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Model                                                                     */
/* ------------------------------------------------------------------------ */

/* Validate *desc, factor the correlation (FP64 Cholesky), build the
 * breadth-first Brownian-bridge schedule and the per-date drift / discount
 * tables, and upload them to the context's device.
 * Errors: PC_EINVAL, PC_ENOTPD, PC_ELIMIT, PC_ENOMEM, PC_ECUDA. */
pc_status pc_model_create(pc_ctx *ctx, const pc_model_desc *desc, pc_model **out);
pc_status pc_model_destroy(pc_model *model);

/* Static facts about a model's path generator. */
typedef struct pc_model_info {
  int32_t d, n_dates, n_hist, t_now;
  int32_t bridge_levels;     /* levels of the bisection tree                      */
  int32_t bridge_stack;      /* bridge values a path holds while dates are made   */
  int32_t philox_blocks;     /* Philox4x32-10 evaluations for all dates of a path  */
  int32_t box_muller_pairs;  /* Box-Muller transforms for all dates of a path      */
} pc_model_info;

/* Fill *info for `model` (host only, no device work).  Errors: PC_EINVAL. */
pc_status pc_model_query(const pc_model *model, pc_model_info *info);

/* ------------------------------------------------------------------------ */
/* Payoff programs                                                           */
/* ------------------------------------------------------------------------ */

/* Load a payoff expression: decode `bytecode` (n_words words, format above),
 * check stack discipline and types (Fig. 3), bind template variables to
 * template_params[0..n_params-1] (the template environment delta of Sec. 2),
 * fold every payoff(t, p1', p2') to +d, -d or 0 for the two-party view
 * (p1, p2) of Fig. 3, and upload the executable form to the device.
 * consts[0..n_consts-1] are the real literals.  Requires a real result.
 * Errors: PC_EINVAL, PC_EBYTECODE, PC_ETPARAM, PC_ELIMIT, PC_ENOMEM, PC_ECUDA. */
pc_status pc_load_payoff(pc_ctx *ctx, const uint32_t *bytecode, size_t n_words,
                         const double *consts, size_t n_consts,
                         const int32_t *template_params, size_t n_params,
                         int32_t p1, int32_t p2, pc_contract **out);
pc_status pc_contract_destroy(pc_contract *contract);
/* Load n programs in one call (a portfolio): program i is words
 * [word_off[i], word_off[i+1]), real literals [const_off[i], const_off[i+1])
 * and template parameters [param_off[i], param_off[i+1]) of the
 * concatenated arrays (offset arrays of n + 1 entries, non-decreasing; a
 * NULL array with all-zero extents may be passed for consts and params),
 * each loaded as pc_load_payoff with the view (p1, p2) into out[i].  On an
 * error no contract is left loaded (out untouched) and the message names
 * the program.  Errors: as pc_load_payoff. */
pc_status pc_load_payoffs(pc_ctx *ctx, size_t n, const uint32_t *words, const size_t *word_off,
                          const double *consts, const size_t *const_off, const int32_t *params,
                          const size_t *param_off, int32_t p1, int32_t p2, pc_contract **out);

/* Host-only: the checks of pc_load_payoff without a context or device.
 * Fills *info (may be NULL).  Errors as pc_load_payoff. */
pc_status pc_verify_payoff(const uint32_t *bytecode, size_t n_words,
                           const double *consts, size_t n_consts,
                           const int32_t *template_params, size_t n_params,
                           pc_program_info *info);

/* Host-only: assemble the textual S-expression form of IL into bytecode.
 * Grammar: (now) (model L t) (if c a b) (loopif c a b t) (payoff t P P)
 * (texpr t) (neg e) (not e) (add|sub|mult|div|lt|le|eq|and|or|max|min a b)
 * REAL #t #f (nat N); times: INT | $K | (tplus t t); ';' comments.
 * Writes at most cap_words words / cap_consts constants and their counts;
 * on PC_ESYNTAX writes a message into err (err_cap bytes, may be 0).
 * Errors: PC_EINVAL, PC_ESYNTAX, PC_ELIMIT (buffers too small). */
pc_status pc_assemble(const char *text, uint32_t *words, size_t cap_words,
                      size_t *n_words, double *consts, size_t cap_consts,
                      size_t *n_consts, char *err, size_t err_cap);

/* Host-only: cutPayoff (Sec. 4.1) on bytecode.  Every payoff(t, p1', p2')
 * becomes if(t < now, 0, payoff(t, p1', p2')), so a contract loaded once
 * can be priced at any valuation time: with the model's t_now = now the
 * payments before now are dropped (Theorem 5: the result is the value of
 * the cashflows from now on).  Every other instruction is copied; the
 * literal 0.0 is appended to the constants unless one is present.  Writes at
 * most cap_words words / cap_consts constants and their counts.
 * Errors: PC_EINVAL, PC_EBYTECODE (bad opcode or truncated operands),
 * PC_ELIMIT (buffers too small, or more than PC_MAX_PROGRAM input words). */
pc_status pc_cut_payoff(const uint32_t *bytecode, size_t n_words, const double *consts,
                        size_t n_consts, uint32_t *out_words, size_t cap_words,
                        size_t *n_out_words, double *out_consts, size_t cap_consts,
                        size_t *n_out_consts);

/* ------------------------------------------------------------------------ */
/* Pricing                                                                   */
/* ------------------------------------------------------------------------ */

/* Monte Carlo value of `contract` under `model` (both on one context):
 * the average over paths 0..n_paths-1 of the discounted payoff, i.e. of
 * IL[[e]](rho_path, delta, 0, t_now, d, p1, p2) (Fig. 3; by Theorem 1 the
 * discounted sum of the contract's cashflows), and its standard error
 * sqrt(sample variance / n).  Path p draws its normals from Philox4x32-10
 * counter (m >> 2, p_lo, p_hi, 0) under key (seed_lo, seed_hi).  Blocks
 * until done.  n_paths >= 2.
 * Errors: PC_EINVAL, PC_ERANGE, PC_ELIMIT, PC_ECUDA, PC_ETIMEOUT, PC_EDEVICE. */
pc_status pc_price(const pc_model *model, const pc_contract *contract,
                   uint64_t n_paths, uint64_t seed,
                   double *out_price, double *out_stderr);

/* Asynchronous form: enqueue the pricing of paths
 * path_offset .. path_offset+n_paths-1 with Philox stream word `stream` and
 * write {sum x, sum x^2, n} as three doubles to the device buffer d_out.
 * Does not synchronise.  n_paths >= 1.  Runs the same kernels as pc_price;
 * results of runs over disjoint path ranges combine by adding the triples.
 * Errors: PC_EINVAL, PC_ERANGE, PC_ELIMIT, PC_ECUDA. */
pc_status pc_price_async(const pc_model *model, const pc_contract *contract,
                         uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                         uint32_t stream, double *d_out);

/* Parity form: as pc_price_async, and also write the FP32 discounted payoff
 * of path path_offset+i to d_payoffs[i] (device, n_paths floats).  Same
 * kernel code path as pc_price_async with the per-path store enabled. */
pc_status pc_price_paths(const pc_model *model, const pc_contract *contract,
                         uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                         uint32_t stream, double *d_out, float *d_payoffs);

/* Most paths one pc_price_noalloc call may price. */
#define PC_NOALLOC_MAX_PATHS (1ull << 24)

/* pc_price_async for callers that cannot allocate device memory -- for
 * example code running under an allocator or framework that owns all of
 * the GPU's memory, or code that must not call cudaMalloc at this point of
 * its run.  The paper has no counterpart; this is an engineering entry point.
 * It writes the same {sum x, sum x^2, n} triple to the device buffer d_out
 * as pc_price_async would with the context's default settings, but takes
 * the kernel's scratch (per-tile partial sums and work counters) from one
 * fixed device array that the library reserves in every GPU that loads it
 * (4 MiB + 18 KiB, held until the process exits), instead of from memory
 * the context allocates.  pc_create looks the array's device address up for
 * its device, so the array is in place before the first call.  The call
 * makes no cudaMalloc, cudaFree or other allocating call, and the library
 * allocates no host memory in it on success (a failure records its message
 * as pc_last_error does).
 *   - n_paths must be 1..PC_NOALLOC_MAX_PATHS; larger requests fail with
 *     PC_ELIMIT.
 *   - Only the interpreting kernel with the window of dates in shared
 *     memory: programs that look back more than PC_MAX_WINDOW dates fail
 *     with PC_ERANGE, and programs whose per-path state leaves no resident
 *     block fail with PC_ELIMIT, where pc_price_async would keep their
 *     window in HBM.  pc_set_jit and pc_set_window_mode do not apply; the
 *     sums equal pc_price_async's bit for bit (its specialised kernel is
 *     bit-identical to the interpreter).
 *   - Every call shares the one array: calls whose kernels overlap on the
 *     GPU (other streams, other contexts on the same device) race and give
 *     wrong results.  Calls on one stream are ordered and safe.  Each call
 *     zeroes the counters it needs before its kernel starts.
 * Errors: PC_EINVAL, PC_ERANGE, PC_ELIMIT, PC_ECUDA. */
pc_status pc_price_noalloc(const pc_model *model, const pc_contract *contract,
                           uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                           uint32_t stream, double *d_out);

/* ------------------------------------------------------------------------ */
/* Window of simulated dates                                                 */
/* ------------------------------------------------------------------------ */
/* A path keeps the simulated values of its recent dates in a window of
 * `win` dates (a power of two above the program's largest lookback below
 * the newest simulated date, from the load-time analysis).  By default the
 * window lives in shared memory.  Programs whose window does not fit there
 * well -- more than PC_MAX_WINDOW dates, or fewer than 8 resident warps per
 * SM -- are not streamable in shared memory; pc_price, pc_price_async and
 * pc_price_paths then keep the window in HBM instead: one column of
 * win * d float2 slots per thread of the launch (slot-major, coalesced),
 * in a buffer the context grows as needed (see pc_price_info).  Results do
 * not depend on where the window lives.  Portfolio, sensitivity,
 * control-variate and no-allocation pricing keep the shared window (they
 * return PC_ERANGE / PC_ELIMIT for programs that need the HBM window).
 * Not in the paper: its generated code reads a path array (Sec. 6.2). */
#define PC_WINDOW_AUTO    0
#define PC_WINDOW_SHARED  1   /* never use the HBM window */
#define PC_WINDOW_HBM     2   /* always use the HBM window (single-contract pricing) */

/* Placement policy of the context's pricing launches.  Errors: PC_EINVAL. */
pc_status pc_set_window_mode(pc_ctx *ctx, int32_t mode);

typedef struct pc_launch_info {
  int32_t window;              /* dates in the window                       */
  int32_t hbm_window;          /* 1: window in HBM                          */
  int32_t block, grid;         /* launch shape                              */
  uint64_t smem_bytes;         /* dynamic shared memory per block           */
  uint64_t hbm_window_bytes;   /* HBM window buffer this launch uses (0 if shared) */
  uint64_t window_bytes_written_per_path_date;  /* HBM window: 4 d        */
} pc_launch_info;

/* How pc_price would launch (model, contract, n_paths) on this context.
 * Host only apart from occupancy queries.  Errors: as pc_price. */
pc_status pc_price_info(const pc_model *model, const pc_contract *contract, uint64_t n_paths,
                        pc_launch_info *info);

/* ------------------------------------------------------------------------ */
/* Run-time specialised pricing kernels                                      */
/* ------------------------------------------------------------------------ */
/* The paper compiles each contract into its own payoff function (Sec. 6).
 * With pc_set_jit(ctx, 1), pc_price / pc_price_async / pc_price_paths run a
 * kernel specialised to the contract's executable program (compiled at run
 * time by NVRTC on first use for each underlying count, cached on the
 * context by program content -- reloading the same program reuses it --
 * and freed by pc_destroy): the same operations in the same order as the
 * interpreting kernel, without the per-instruction dispatch, with the
 * window of dates in shared memory or in HBM as the launch places it.
 * pc_price_cv and pc_greeks likewise run specialised control-variate and
 * tangent kernels.  Programs of more than PC_JIT_MAX_INSNS executable instructions are not
 * specialised (NVRTC's time grows faster than the program's length: about
 * 20 s for 600 instructions); their launches interpret them.
 * Default: 0 (interpret).  Errors: PC_EINVAL. */
#define PC_JIT_MAX_INSNS 384
pc_status pc_set_jit(pc_ctx *ctx, int32_t enabled);
/* Compile (now) the contract's specialised kernel for the model's
 * underlying count (shared-memory window, pooled sums); does nothing for a
 * program beyond PC_JIT_MAX_INSNS instructions.  Blocks; typically tens
 * of milliseconds to a few seconds.
 * Errors: PC_EINVAL, PC_ECUDA (the compiler's log in pc_last_error). */
pc_status pc_jit_compile(const pc_model *model, const pc_contract *contract);

/* ------------------------------------------------------------------------ */
/* Portfolio pricing                                                         */
/* ------------------------------------------------------------------------ */
/* The paper prices one contract per engine invocation; templating (Sec. 2,
 * Sec. 6.2) is what makes many instruments of one shape cheap to set up.
 * A batch plan prices many such contracts -- uneven program lengths, date
 * counts and path budgets -- in persistent launches, one per group of
 * contracts with the same underlying count and a similar per-path shared-
 * memory footprint.  Work units (a contract and a run of its 64-path tiles)
 * are ordered costliest first and taken by warps from a counter; each
 * contract reduces into its own scratch, so its price and standard error
 * are bit-identical to pc_price(models[i], contracts[i], n_paths[i], seed)
 * with Philox stream word i -- i.e. to pc_price_paths/pc_price_async with
 * stream = i, path_offset = 0.  The launches are captured once into a CUDA
 * graph and replayed by pc_batch_launch. */
typedef struct pc_batch pc_batch;

/* Launch shape of a plan.  block: threads per block preferred for every
 * group (128, 64 or 32; a group whose footprint does not fit falls back to
 * the next smaller size).  unit_split: each warp's fair share of the plan's
 * estimated work is cut into about this many units (>= 1); a contract's
 * unit is its tiles grouped so that the unit's estimated cost is at most
 * that share (at least one tile).  The paths a thread evaluates per unit
 * are 2 x tiles per unit. */
typedef struct pc_batch_config {
  int32_t block;
  int32_t unit_split;
} pc_batch_config;

typedef struct pc_batch_info {
  uint64_t n_contracts;
  uint64_t n_tiles;          /* 64-path tiles over all contracts            */
  uint64_t n_units;          /* work units under the current config         */
  int32_t n_groups;          /* persistent launches per replay              */
  int32_t tuned;             /* 1 after pc_batch_tune                       */
  pc_batch_config config;    /* current launch shape                        */
  double paths_per_thread;   /* mean paths a thread evaluates per unit      */
  double last_ms;            /* device time of the last timed replay (tune) */
  int32_t n_specialised;     /* contracts on their own run-time specialised
                                kernel (with pc_set_jit: the costliest)    */
} pc_batch_info;

/* Build a plan over n contracts: contract i is priced against models[i]
 * with n_paths[i] paths (2 .. 2^40) on Philox stream word i under `seed`.
 * With the context's pc_set_jit on, the costliest contracts (up to 160, and
 * until 80 % of the estimated work) are priced by their run-time
 * specialised kernels, each its own branch of the replay, the rest by the
 * interpreting group kernels; the results are the same bits either way
 * (compiling takes a few tens of ms per new program, cached per context).
 * All models and contracts must belong to one context and stay alive until
 * pc_batch_destroy.  config may be NULL (block 128, unit_split 128).
 * Allocates the plan's device memory (per-contract arguments, units,
 * reduction scratch, outputs) and instantiates its graph.
 * Errors: PC_EINVAL (null, empty, mixed contexts, n_paths out of range),
 * PC_ERANGE (a program reads a label or date outside its model), PC_ELIMIT
 * (a contract's per-path state exceeds shared memory), PC_ENOMEM, PC_ECUDA. */
pc_status pc_batch_create(size_t n, const pc_model *const *models,
                          const pc_contract *const *contracts,
                          const uint64_t *n_paths, uint64_t seed,
                          const pc_batch_config *config, pc_batch **out);

/* Autotuner: times every candidate launch shape (block 128 / 64, unit_split
 * 8 / 32 / 128) over `reps` replays each (>= 1, after one warm-up replay)
 * with CUDA events on the context's stream, keeps the fastest and
 * re-instantiates the graph with it.  Results of the plan are unchanged by
 * the shape.  Blocks until done.  Errors: as pc_batch_launch. */
pc_status pc_batch_tune(pc_batch *plan, int32_t reps);

/* Replay the plan's graph on the context's stream (asynchronous).
 * Errors: PC_EINVAL, PC_ECUDA. */
pc_status pc_batch_launch(pc_batch *plan);

/* Wait for the last replay and return out_price[i], out_stderr[i] (host,
 * [n] each); out_sums (nullable, host [3n]) receives each contract's
 * (sum x, sum x^2, n) for merging partial runs across processes.
 * Errors: PC_ETIMEOUT, PC_EDEVICE, PC_ECUDA. */
pc_status pc_batch_results(pc_batch *plan, double *out_price, double *out_stderr,
                           double *out_sums);

pc_status pc_batch_query(const pc_batch *plan, pc_batch_info *info);

/* Launch arrangement of a plan's replay.  enabled = 0 (the default): one
 * persistent launch per (underlying count, power-of-two class of per-path
 * shared words) group, as parallel branches of the graph, each kernel
 * specialised to its count and sized for its group's footprint.
 * enabled = 1: one persistent launch for every contract (one kernel for all
 * underlying counts, at the register bound of the four-underlying
 * generator, sized for the largest footprint of all), units ordered
 * costliest first over the whole portfolio.  Re-instantiates the graph with
 * the current launch shape (pc_batch_tune may be run again); results are
 * the same either way.  Errors: PC_EINVAL, PC_ELIMIT (the largest footprint
 * does not fit one launch; the plan keeps its grouping), PC_ECUDA. */
pc_status pc_batch_set_single_launch(pc_batch *plan, int32_t enabled);
pc_status pc_batch_destroy(pc_batch *plan);

/* One-shot portfolio pricing: pc_batch_create with the default shape,
 * one replay, pc_batch_results, pc_batch_destroy.  Blocks until done.
 * Errors: as pc_batch_create and pc_batch_results. */
pc_status pc_price_batch(size_t n, const pc_model *const *models,
                         const pc_contract *const *contracts,
                         const uint64_t *n_paths, uint64_t seed,
                         double *out_price, double *out_stderr);

/* Pathwise sensitivities: price, delta_l = d price / d S0[l] and
 * vega_l = d price / d sigma[l] (l < d) from the derivative of each path's
 * payoff through the GBM map (if / loopif decisions held fixed; valid for
 * payoffs that are Lipschitz in the path).  Tangent (forward) mode, one
 * launch per underlying on the same paths as pc_price with this seed.
 * out_delta, out_vega: [d]; out_se: [1+2d] -- out_se[0] is the price's
 * standard error, out_se[1+l] delta_l's, out_se[1+d+l] vega_l's.
 * Blocks until done.  Errors: as pc_price. */
pc_status pc_greeks(const pc_model *model, const pc_contract *contract,
                    uint64_t n_paths, uint64_t seed, double *out_price,
                    double *out_delta, double *out_vega, double *out_se);

/* The same sensitivities by the chain rule in reverse (adjoint mode): one
 * launch gives the price and every underlying's delta and vega.  Each
 * path's payoff program records a tape of its real arithmetic (decisions
 * held fixed as above) and the path state it reads at each observed date
 * (S and X = L W of the read underlying); a reverse sweep of the tape gives
 * d payoff / d S0[l] = sum over reads of the adjoint times S / S0[l], and
 * d / d sigma[l] = sum of the adjoint times S (X - sigma[l] tau).  The paper
 * has no sensitivities; this is the pathwise method (Glasserman, Monte
 * Carlo Methods in Financial Engineering, Sec. 7.2) on the IL semantics of
 * Fig. 3.  Same paths as pc_price with this seed.  The tape lives in a
 * context buffer of grid x warps x (bound on the program's tape entries)
 * x 776 bytes, grown as needed; programs keep their window of dates in
 * shared memory (no HBM window: PC_ERANGE / PC_ELIMIT as pc_price_noalloc).
 * Outputs as pc_greeks.  Blocks until done.  Errors: as pc_price, and
 * PC_ELIMIT for a tape bound above 2^24 entries. */
pc_status pc_greeks_adjoint(const pc_model *model, const pc_contract *contract,
                            uint64_t n_paths, uint64_t seed, double *out_price,
                            double *out_delta, double *out_vega, double *out_se);

/* Asynchronous form on the context's stream, paths path_offset.. of Philox
 * stream `stream`: d_out (device, 2 (1 + 2d) + 1 doubles) receives the sums
 * and sums of squares of (payoff, delta_0..delta_{d-1}, vega_0..vega_{d-1})
 * per path, interleaved (sum, sum of squares) per quantity, then n_paths. */
pc_status pc_greeks_adjoint_async(const pc_model *model, const pc_contract *contract,
                                  uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                                  uint32_t stream, double *d_out);

/* ------------------------------------------------------------------------ */
/* Learned control variate: network                                          */
/* ------------------------------------------------------------------------ */
/* Not in the paper (an extension of its Monte Carlo valuation).  A
 * multilayer perceptron widths[0] -> ... -> widths[L]: softplus hidden
 * layers, linear output; BF16 weights and activations, FP32 accumulation
 * on the tensor cores, FP32 master weights updated by Adam.  Trained on the
 * engine's own prices and sensitivities to give hedge ratios for the
 * control variate below.  Samples are rows: x [n, widths[0]],
 * y and targets [n, widths[L]], FP32.  Parameters, "unpadded layout": for
 * each layer l, W_l [widths[l+1], widths[l]] row-major, then b_l
 * [widths[l+1]].  Results are deterministic (fixed-order reductions). */
typedef struct pc_mlp pc_mlp;

typedef struct pc_mlp_info {
  int32_t n_layers;          /* L                                            */
  int32_t widths[9];         /* widths[0..L]                                 */
  uint64_t n_params;         /* floats in the unpadded layout                */
  uint64_t max_batch;        /* rows per forward / gradient call             */
  uint64_t steps;            /* Adam steps taken                             */
} pc_mlp_info;

/* widths: n_widths = L + 1 (2..9) entries; widths[0] and widths[L] in
 * 1..64, hidden widths multiples of 64 up to 1024.  max_batch: rows per
 * call (>= 1).  Weights start uniform in +-1/sqrt(fan-in) from `seed`.
 * Errors: PC_EINVAL, PC_ENOMEM, PC_ECUDA. */
pc_status pc_mlp_create(pc_ctx *ctx, const int32_t *widths, int32_t n_widths, uint64_t max_batch,
                        uint64_t seed, pc_mlp **out);
pc_status pc_mlp_destroy(pc_mlp *net);
pc_status pc_mlp_query(const pc_mlp *net, pc_mlp_info *info);
/* Host arrays of n = info.n_params floats (unpadded layout).  set resets
 * the Adam moments and step count. */
pc_status pc_mlp_set_params(pc_mlp *net, const float *params, size_t n);
pc_status pc_mlp_get_params(const pc_mlp *net, float *params, size_t n);
/* d_y [n, widths[L]] = network(d_x [n, widths[0]]), device pointers, any n
 * (processed in max_batch chunks).  Asynchronous on the context's stream. */
pc_status pc_mlp_forward(pc_mlp *net, const float *d_x, size_t n, float *d_y);
/* Loss (1/n) sum_b sum_j w_j (y_bj - t_bj)^2 of the n <= max_batch samples
 * (device d_x, d_t; host w [widths[L]]) and its gradient with respect to
 * every parameter, d_grads (device, unpadded layout, nullable).  No update.
 * Blocks until done; *out_loss (host). */
pc_status pc_mlp_gradients(pc_mlp *net, const float *d_x, const float *d_t, const float *w,
                           size_t n, float *d_grads, double *out_loss);
/* Product kernels of the network.  PC_MLP_GEMM_AUTO (the default): the
 * forward products run on the tcgen05 tensor cores (TMA-staged operands,
 * TMEM accumulators) where the device has them, the backward products and
 * every product elsewhere on the warp-level BF16 MMA kernel;
 * PC_MLP_GEMM_MMA_SYNC: the warp-level kernel for every product.  Both
 * accumulate in FP32 (results differ by summation order only).  Changing
 * the choice re-captures the training step.  pc_mlp_gemm_info:
 * *tensor_cores = 1 when the forward products use tcgen05.  A tensor-core
 * product whose bounded wait expires sets a status that the next blocking
 * call on the network (pc_mlp_gradients, pc_mlp_train, pc_cv_tables)
 * reports as PC_ETIMEOUT.  Errors: PC_EINVAL. */
#define PC_MLP_GEMM_AUTO 0
#define PC_MLP_GEMM_MMA_SYNC 1
pc_status pc_mlp_set_gemm(pc_mlp *net, int32_t kind);
pc_status pc_mlp_gemm_info(const pc_mlp *net, int32_t *tensor_cores);
/* `steps` Adam steps (lr; b1 0.9, b2 0.999, eps 1e-8) on minibatches of
 * `batch` rows (1..max_batch) drawn with replacement from the n_data rows of
 * d_x / d_t by Philox4x32-10 under `seed` and the step number.  One step is
 * captured once into a CUDA graph and replayed.  Blocks until done;
 * *out_loss = loss of the last minibatch (before its update).
 * Errors: PC_EINVAL, PC_ECUDA, PC_ETIMEOUT. */
pc_status pc_mlp_train(pc_mlp *net, const float *d_x, const float *d_t, size_t n_data,
                       const float *w, size_t batch, int32_t steps, float lr, uint64_t seed,
                       double *out_loss);

/* ------------------------------------------------------------------------ */
/* Learned control variate: delta-hedge estimator                            */
/* ------------------------------------------------------------------------ */
/* For a worst-of autocallable contract (payments decided at the model's
 * dates t_1..t_n by worst_k = min_i S_i(t_k) / ref_i: called at t_k < t_n
 * when worst_k >= call_level, knock-in when some worst_k <= ki_level) the
 * pricing kernel adds to each path's payoff X the discounted gains of a
 * hedge held over [t_k, t_{k+1}] while the contract is alive,
 *   M = sum_k alive_k sum_i Delta_i(k) (D_{k+1} S_i(t_{k+1}) - D_k S_i(t_k)),
 * and reports Y = X - beta M - beta2 M2.  The D S_i are martingales and
 * every Delta_i(k) depends only on the path up to t_k, so E[M] = 0: Y is
 * unbiased for any hedge ratios and any fixed betas, and its variance is
 * small when the ratios are close to the contract's sensitivities.  The
 * optional second-order term (use_gamma) is
 *   M2 = sum_{k>=1} alive_k 1/2 sum_ij Gamma_ij(k) (X_i X_j - E_k[X_i X_j]),
 * X_i = D_{k+1} S_i(t_{k+1}) - D_k S_i(t_k), with E_k[X_i X_j] =
 * D_k^2 S_i S_j (exp(rho_ij sigma_i sigma_j (tau_{k+1} - tau_k)) - 1) in
 * closed form and Gamma from the slopes of the table's interpolant
 * (Gamma_ij = (s_ij / (h_j S_j) + s_ji / (h_i S_i)) / 2, s_ij = d Delta_i /
 * d u_j), so E[M2] = 0 as well.  Hedge ratios at t_k (k >= 1) come from a
 * table over y = ln S per date and knock-in state, read by multilinear
 * interpolation (per axis u = clamp((y - lo) / h, 0, G - 1),
 * a = min(floor(u), G - 2), f = u - a), at t_0 from delta0.  Tables are
 * filled by a trained network (pc_cv_tables) or by the caller.  Table
 * layout (floats, 16-byte aligned): [(k - 1) * 2 + ki][node][4] with the d
 * ratios first in each group of four, node = ((a_0 G + a_1) G + a_2) (axis
 * 0 slowest), k = 1..n-1, ki = knock-in flag.
 * Not in the paper (an extension of its Monte Carlo valuation). */
#define PC_CV_MAX_DATES 32

typedef struct pc_cv_desc {
  int32_t d;                 /* underlyings, 1..3 (the model's d)            */
  int32_t n;                 /* observation dates (the model's dates), 1..32 */
  int32_t grid;              /* table nodes per axis G, 2..64                */
  float ref[3];              /* worst = min_i S_i / ref_i                    */
  float call_level, ki_level, coupon;
  float lo[PC_CV_MAX_DATES][3];  /* table axes over ln S: row k - 1 = date k */
  float h[PC_CV_MAX_DATES][3];
  float delta0[3];           /* hedge ratios at t_0                          */
  float beta;                /* Y = X - beta M - beta2 M2 (pc_cv_grid: 1)    */
  float beta2;               /* (pc_cv_grid: 1)                              */
  int32_t use_gamma;         /* 1: include M2 (pc_cv_grid: 0)                */
  int32_t delta0_on_device;  /* 1: the pricing reads delta0 from the device,
                                the 4 floats after the tables (set by
                                pc_cv_tables_async); 0: delta0 above      */
} pc_cv_desc;

/* Training labels of the learned control variate from the engine's prices
 * of sampled states: row c of out (width floats, host) = the price at the
 * state, then the central-difference hedge ratios on common random numbers
 * (P(S_i (1 + bump)) - P(S_i (1 - bump))) / (2 bump S_i), i < d, then zeros.
 * prices: [(2d + 1) x n] doubles, row 0 at the state, rows 1 + 2i and 2 + 2i
 * with S_i bumped up and down; spots: [n x d].  Errors: PC_EINVAL. */
pc_status pc_cv_labels(size_t n, int32_t d, const double *prices, const double *spots, double bump,
                       int32_t width, float *out);

/* Fill d, n, grid, lo and h from the model: axis i at date k is centred on
 * ln S0_i + (r - sigma_i^2 / 2) tau_k with half-width width_sd sigma_i
 * sqrt(tau_k).  The caller sets ref, the levels, coupon (and delta0 when it
 * fills the tables itself).  Errors: PC_EINVAL, PC_ELIMIT (d > 3 or more
 * than PC_CV_MAX_DATES dates). */
pc_status pc_cv_grid(const pc_model *model, int32_t grid, float width_sd, pc_cv_desc *desc);
/* Floats of the tables of desc: (n - 1) * 2 * grid^d * 12.  Table (k - 1) * 2
 * + knock-in holds date k's nodes, node index sum_i a_i grid^(d-1-i), 12
 * floats each: the hedge ratios Delta_0..2, then their slopes along the grid
 * axes s_ij = d Delta_i / d u_j at 3 + 3 i + j (zero beyond d).  A path at
 * grid coordinate u (u_i = (ln S_i - lo_i) / h_i, clamped to [0, grid - 1])
 * takes the nearest node a = floor(u + 1/2): Delta_i = Delta_i(a) + sum_j
 * s_ij(a) (u_j - a_j), and gamma_ij = s_ij / (h_j S_j) symmetrised. */
pc_status pc_cv_table_size(const pc_cv_desc *desc, size_t *floats);
/* Evaluate the network (16 inputs, outputs value and hedge ratios) at every
 * table node and at the spot and write d_tables (device, cap_floats: the
 * ratios from the network, the slopes as central differences of the
 * neighbouring nodes' ratios, one-sided on the grid's faces) and
 * desc->delta0.  Network inputs of a state (date k, y = ln S, knock-in):
 * y_i - ln ref_i (i < 3, 0 beyond d), sigma_i (i < 3), the correlation of
 * underlyings 0 and 1 (0 if d = 1), r, tau_{k+1} - tau_k, (n - k) / 5,
 * k / 5, knock-in, coupon, call_level, ki_level, 1.  Blocks until done.
 * Errors: PC_EINVAL (widths other than 16 in / 5 out, cap too small). */
pc_status pc_cv_tables(pc_mlp *net, const pc_model *model, pc_cv_desc *desc, float *d_tables,
                       size_t cap_floats);
/* pc_cv_tables without the wait: the build is enqueued on the context's
 * stream and delta0 is written on the device, to the 4 floats after the
 * tables (cap_floats >= pc_cv_table_size + 4), where pc_price_cv reads it:
 * sets desc->delta0_on_device = 1 and zeroes desc->delta0.  A bounded wait
 * that expires in the build is reported (PC_ETIMEOUT) by the next blocking
 * call on the network (pc_cv_tables, pc_mlp_forward, pc_mlp_gradients,
 * pc_mlp_train).  Errors: as pc_cv_tables. */
pc_status pc_cv_tables_async(pc_mlp *net, const pc_model *model, pc_cv_desc *desc, float *d_tables,
                             size_t cap_floats);
/* Price with the control variate: out[0..3] (host) = price and standard
 * error of Y = X - beta M - beta2 M2 (betas from desc), then of X on the
 * same paths (pc_price's estimate with this seed).  d_tables: device
 * tables laid out as above.  Blocks until done.
 * Errors: as pc_price; PC_EINVAL for a desc that does not match the model. */
pc_status pc_price_cv(const pc_model *model, const pc_contract *contract, const pc_cv_desc *desc,
                      const float *d_tables, uint64_t n_paths, uint64_t seed, double *out);
/* Pilot run: the variance-minimising betas measured on n_paths (>= 16)
 * paths under `seed` (use an independent seed or stream for the priced run
 * so that its betas are fixed): beta[0] (and beta[1] with use_gamma, else
 * 0) solve Cov([M, M2]) beta = Cov(X, [M, M2]).  Blocks until done.
 * Errors: as pc_price_cv. */
pc_status pc_cv_beta(const pc_model *model, const pc_contract *contract, const pc_cv_desc *desc,
                     const float *d_tables, uint64_t n_paths, uint64_t seed, double *beta);

/* ------------------------------------------------------------------------ */
/* Parity probes (same device functions as the pricing kernel)               */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 on the device: for i < n, out[4i..4i+3] = Philox of counter
 * ctr[4i..4i+3] under key (key0, key1).  ctr, out: device uint32 arrays. */
pc_status pc_debug_philox(pc_ctx *ctx, const uint32_t *d_ctr, uint32_t key0,
                          uint32_t key1, uint32_t *d_out, size_t n);

/* Simulated path values: d_S[(i*d + l)*(n_dates+1) + o] = S_l at ordinal o
 * (o = 0..n_dates) of path path_offset+i, FP32, device.  Same path
 * generator as the pricing kernel. */
pc_status pc_debug_paths(const pc_model *model, uint64_t n_paths,
                         uint64_t path_offset, uint64_t seed, uint32_t stream,
                         float *d_S);

/* Failure injection for tests of the error paths (no device fault is
 * involved): the context's next `count` device allocations fail as if the
 * device were out of memory (the call reports PC_ENOMEM; nothing is
 * allocated or leaked).  count = 0 ends the injection. */
pc_status pc_debug_fail_allocations(pc_ctx *ctx, int32_t count);

/* Write `value` into the context's device status word (as a kernel that
 * clamped an access would): the next blocking call reports PC_EDEVICE and
 * clears it.  Blocks until written. */
pc_status pc_debug_set_status(pc_ctx *ctx, int32_t value);

/* Paths a lane of the context's specialised pricing kernels for programs
 * that read no date behind the frontier: pairs = 1 (two paths a lane), 2
 * (four: the per-op bridge schedule and the per-instruction control serve
 * twice the paths, with twice the per-thread bridge stack) or 0, the
 * default (two pairs when the model has at least 64 dates, else one).  The
 * per-path values and sums are the same either way; the kernels are cached
 * per choice.  Errors: PC_EINVAL. */
pc_status pc_debug_set_jit_pairs(pc_ctx *ctx, int32_t pairs);

/* Resident 128-thread blocks per SM the register bound of the context's
 * specialised control-variate kernels is set for (1..16), or 0 for the
 * default (5).  The values
 * are the same under any bound; the kernels are cached per choice.
 * Errors: PC_EINVAL. */
pc_status pc_debug_set_cv_min_blocks(pc_ctx *ctx, int32_t blocks);

/* Failure test of the network's tensor-core product: while `on`, its TMA
 * producer withholds the copies of the first k-chunk, so the MMA issuer's
 * and the producer's bounded mbarrier waits expire (after about 10 ms
 * instead of the normal second); the kernel sets the network's status word,
 * stops issuing, lets the copies it did issue land, frees its tensor memory
 * and returns.  The next blocking network call (pc_mlp_gradients,
 * pc_mlp_train) reports PC_ETIMEOUT and clears the word.  Drops the
 * network's captured graphs. */
pc_status pc_debug_mlp_withhold_tma(pc_mlp *net, int32_t on);

/* Per-path probe of pc_greeks for one underlying: writes (payoff,
 * d payoff / d S0[underlying], d payoff / d sigma[underlying]) of path
 * path_offset+i to d_paths[3i..3i+2] (device floats) and the six sums
 * (value, value^2, delta, delta^2, vega, vega^2) then n to d_out[0..6]
 * (device doubles).  Asynchronous on the context's stream. */
pc_status pc_debug_greeks_paths(const pc_model *model, const pc_contract *contract,
                                uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                                int32_t underlying, double *d_out, float *d_paths);

/* Per-path probe of pc_greeks_adjoint: path path_offset+i writes (payoff,
 * delta_0..delta_{d-1}, vega_0..vega_{d-1}) to d_paths[(1+2d)i ..] (device
 * floats); d_out as pc_greeks_adjoint_async.  Asynchronous on the
 * context's stream. */
pc_status pc_debug_adjoint_paths(const pc_model *model, const pc_contract *contract,
                                 uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                                 double *d_out, float *d_paths);

/* Per path i < n_paths (paths 0.., Philox stream 0): d_xm[3i] = payoff X,
 * d_xm[3i + 1] = hedge gain M, d_xm[3i + 2] = second-order gain M2 of
 * pc_price_cv (device floats; M2 computed whatever desc->use_gamma).
 * Asynchronous on the context's stream. */
pc_status pc_debug_cv_paths(const pc_model *model, const pc_contract *contract, const pc_cv_desc *desc,
                            const float *d_tables, uint64_t n_paths, uint64_t seed, float *d_xm);

/* Host-only: generate and compile (NVRTC, sm_103a) a specialised kernel of
 * a program for d underlyings, without loading it; *cubin_bytes receives
 * the size of the result.  kind: 0 the pricing kernel, 1 its per-path
 * variant, 2 and 3 those two with the window of dates in HBM, 16 + m the
 * control-variate kernel of mode m (bits: 1 per-path outputs, 2
 * second-order term, 4 pilot sums; d <= 3), 32 the sensitivity kernel and
 * 33 its per-path variant.  Errors: as
 * pc_verify_payoff; PC_EINVAL for another kind; PC_ECUDA with the
 * compiler's log. */
pc_status pc_debug_jit_compile(const uint32_t *bytecode, size_t n_words, const double *consts,
                               size_t n_consts, const int32_t *template_params, size_t n_params,
                               int32_t p1, int32_t p2, int32_t d, int32_t kind, size_t *cubin_bytes);

/* Host-only: the CUDA C++ source that pc_debug_jit_compile hands to NVRTC
 * for the same arguments (it includes the library's device headers by
 * name).  *len receives its length; the text and a terminating NUL are
 * written to out when cap > *len (out may be NULL to query the length).
 * Identifies the kernel a profile was taken on.  Errors: as
 * pc_debug_jit_compile. */
pc_status pc_debug_jit_source(const uint32_t *bytecode, size_t n_words, const double *consts,
                              size_t n_consts, const int32_t *template_params, size_t n_params,
                              int32_t p1, int32_t p2, int32_t d, int32_t kind, char *out, size_t cap,
                              size_t *len);

/* Host-only: the executable form pc_load_payoff would run for this program:
 * 4 words per instruction (opcode | A << 8, then three operand words), then
 * the program's constant pool (float bits).  Writes *n_insn and *n_pool,
 * and the 4 * n_insn + n_pool words to out when cap_words allows.
 * Errors: as pc_load_payoff; PC_ELIMIT if cap_words is too small. */
pc_status pc_debug_program(const uint32_t *bytecode, size_t n_words,
                           const double *consts, size_t n_consts,
                           const int32_t *template_params, size_t n_params,
                           int32_t p1, int32_t p2, uint32_t *out, size_t cap_words,
                           size_t *n_insn, size_t *n_pool);

/* Host-only: the date-ordered bridge schedule pc_model_create builds for
 * *desc: date_ops[0..n_dates+1] (ops of date t are date_ops[t] ..
 * date_ops[t+1]-1) and 6 words per op (wl, wr, sd as float bits; node
 * number; flags << 16; date ordinal).  Writes at most cap_ops ops.
 * Errors: as pc_model_create's validation; PC_ELIMIT if cap_ops is small. */
pc_status pc_debug_bridge(const pc_model_desc *desc, int32_t *date_ops, uint32_t *ops,
                          size_t cap_ops, size_t *n_ops);

#ifdef __cplusplus
}
#endif
#endif /* PC_H */
