// pc_adjoint_api.cpp -- pc_greeks_adjoint and its asynchronous and per-path
// forms: the launch set-up of the adjoint kernel (pc_adjoint.cuh).
//
// Layout of a thread's shared region: two physical slots per program value
// (the value and its tape entry number), the bridge stack, the window of
// S and the window of X = L W.  The tape bound comes from the load-time
// walk of the program (TimeWalk::entries); the tape buffer is the
// context's, grown to grid x warps per block regions of that bound.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "pc_handles.h"

using namespace pc;

namespace {

// Bytes of one warp's tape region for `emax` entries.
size_t tape_region_bytes(int64_t emax) {
  return size_t(emax) * (32 * (sizeof(float4) + sizeof(float2)) + sizeof(int2));
}

// Tape memory above which the launch is given fewer resident warps.
constexpr size_t kTapeCapBytes = size_t(8) << 30;

pc_status run_adjoint(const pc_model *m, const pc_contract *k, uint64_t n_paths, uint64_t offset,
                      uint64_t seed, uint32_t stream, double *d_out, float *d_paths) {
  Launch L;
  pc_status s = prepare(m, k, n_paths, offset, seed, stream, L, false);
  if (s != PC_OK) return s;
  pc_ctx *c = m->ctx;
  const ModelHost &H = m->H;
  const int d = H.d;
  // the tape bound of this program on this model's dates
  const char *why = "";
  auto on_fail = [&](pc_status st, int64_t, int64_t) {
    why = st == PC_ELIMIT ? "program too long to analyse (loop trip counts)"
                          : "a model or payoff time is outside the model's grid";
  };
  TimeWalk<decltype(on_fail)> walk{k->prog.code.data(), H.t_now, H.n, H.n_hist, on_fail};
  walk.run(0, k->prog.code.size(), 0);
  if (walk.st != PC_OK) return fail(walk.st, why);
  const int64_t emax = std::max<int64_t>(walk.entries, 1);
  if (emax > (int64_t(1) << 24)) return fail(PC_ELIMIT, "adjoint tape bound above 2^24 entries per path");
  Layout lay = L.args.lay;
  lay.stack = 2 * k->prog.frame_slots;
  lay.off_bstack = lay.stack;
  lay.off_cache = lay.off_bstack + H.bstack * d;
  lay.off_win = lay.off_cache;
  lay.off_xwin = lay.off_win + lay.win * d;
  lay.words = lay.off_xwin + lay.win * d;
  int block = 0, best_warps = 0;
  size_t smem = 0;
  for (int b = kBlock; b >= 32; b /= 2) {
    const size_t sm = price_smem_bytes(k->prog.code.size(), pool_padded(k->prog), lay.words, b);
    if (sm + kStaticSmemReserve > size_t(c->max_smem)) continue;
    const int warps = adjoint_blocks_per_sm(d, b, sm) * (b / 32);
    if (warps > best_warps) {
      block = b;
      best_warps = warps;
      smem = sm;
    }
  }
  if (!block) return fail(PC_ELIMIT, "program + per-path state with the adjoint tape slots exceed shared memory");
  const int wpb = block / 32;
  const uint64_t need = (L.args.n_tiles + wpb - 1) / wpb;
  int grid = int(std::min<uint64_t>(uint64_t(c->sm_count) * (best_warps / wpb), need));
  const size_t region = tape_region_bytes(emax);
  if (size_t(grid) * wpb * region > kTapeCapBytes)
    grid = int(std::max<size_t>(1, kTapeCapBytes / (size_t(wpb) * region)));
  const size_t bytes = size_t(grid) * wpb * region;
  if (bytes > c->tape_cap) {
    CU(cudaStreamSynchronize(c->stream), "sync");
    if (c->d_tape) cudaFree(c->d_tape);
    c->d_tape = nullptr;
    c->tape_cap = 0;
    CU(ctx_malloc(c, &c->d_tape, bytes), "adjoint tape");
    c->tape_cap = bytes;
  }
  const size_t regions = size_t(grid) * wpb;
  TapeArgs t;
  t.emax = int32_t(emax);
  char *base = static_cast<char *>(c->d_tape);
  t.part = reinterpret_cast<float4 *>(base);
  t.adj = reinterpret_cast<float2 *>(base + regions * size_t(emax) * 32 * sizeof(float4));
  t.ids = reinterpret_cast<int2 *>(base + regions * size_t(emax) * 32 * (sizeof(float4) + sizeof(float2)));
  // reduction: 2 (1 + 2d) doubles per tile; chunk partials within the
  // control block (kMaxChunks x 8 doubles)
  const int width = 2 * (1 + 2 * d);
  PriceArgs a = L.args;
  a.lay = lay;
  a.width = width;
  reduction_chunks(a.n_tiles, a.chunk_tiles, a.n_chunks);
  const uint32_t max_chunks = uint32_t(kMaxChunks * 8 / width);
  if (a.n_chunks > max_chunks) {
    a.chunk_tiles = uint32_t((a.n_tiles + max_chunks - 1) / max_chunks);
    a.n_chunks = uint32_t((a.n_tiles + a.chunk_tiles - 1) / a.chunk_tiles);
  }
  s = ensure_partials(c, size_t(a.n_tiles) * size_t(width));
  if (s != PC_OK) return s;
  a.tile_partials = c->d_partials;
  a.control = c->d_control;
  a.out = d_out;
  a.out_paths = d_paths;
  CU(cudaSetDevice(c->device), "cudaSetDevice");
  if (c->jit && adjoint_jit_eligible(k)) {
    // the program's run-time specialised adjoint kernel (same arguments,
    // block and tape regions; at most the interpreter's grid)
    cudaKernel_t jk = nullptr;
    s = jit_kernel(k, d, kJitAdjoint + (d_paths ? 1 : 0), block, jk);
    if (s != PC_OK) return s;
    const void *kern = reinterpret_cast<const void *>(jk);
    int nb = 0;
    CU(jit_occupancy(c, kern, block, smem, nb), "jit occupancy");
    if (nb >= 1) {
      const int jgrid = std::min(grid, c->sm_count * nb);
      void *args[] = {&a, &t};
      CU(cudaLaunchKernel(kern, dim3(jgrid), dim3(block), args, smem, c->stream), "specialised adjoint kernel");
      return PC_OK;
    }
  }
  CU(launch_adjoint(a, t, grid, block, smem, c->stream), "adjoint kernel");
  return PC_OK;
}

}  // namespace

extern "C" {

pc_status pc_greeks_adjoint_async(const pc_model *m, const pc_contract *k, uint64_t n_paths,
                                  uint64_t path_offset, uint64_t seed, uint32_t stream, double *d_out) {
  if (!m || !k || !d_out) return fail(PC_EINVAL, "null argument");
  return run_adjoint(m, k, n_paths, path_offset, seed, stream, d_out, nullptr);
}

pc_status pc_greeks_adjoint(const pc_model *m, const pc_contract *k, uint64_t n_paths, uint64_t seed,
                            double *out_price, double *out_delta, double *out_vega, double *out_se) {
  if (!m || !k || !out_price || !out_delta || !out_vega || !out_se) return fail(PC_EINVAL, "null argument");
  if (n_paths < 2) return fail(PC_EINVAL, "n_paths must be >= 2 for a standard error");
  pc_ctx *c = m->ctx;
  const int d = m->H.d;
  pc_status s = run_adjoint(m, k, n_paths, 0, seed, 0, c->d_gout, nullptr);
  if (s != PC_OK) return s;
  const int width = 2 * (1 + 2 * d);
  double h[PC_MAX_UNDERLYINGS * 8], st[5];
  CU(cudaMemcpyAsync(h, c->d_gout, size_t(width + 1) * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
     "result copy");
  CU(cudaMemcpyAsync(st, c->d_res, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "status copy");
  s = wait_stream(c);
  if (s != PC_OK) return s;
  int32_t status;
  std::memcpy(&status, &st[4], 4);
  s = check_status(c, status);
  if (s != PC_OK) return s;
  const double n = double(n_paths);
  auto mean_se = [&](int j, double &mean, double &se) {
    mean = h[2 * j] / n;
    se = std::sqrt(std::max(0.0, (h[2 * j + 1] - n * mean * mean) / (n - 1.0)) / n);
  };
  mean_se(0, *out_price, out_se[0]);
  for (int l = 0; l < d; ++l) {
    mean_se(1 + l, out_delta[l], out_se[1 + l]);
    mean_se(1 + d + l, out_vega[l], out_se[1 + d + l]);
  }
  return PC_OK;
}

pc_status pc_debug_adjoint_paths(const pc_model *m, const pc_contract *k, uint64_t n_paths,
                                 uint64_t path_offset, uint64_t seed, double *d_out, float *d_paths) {
  if (!m || !k || !d_out || !d_paths) return fail(PC_EINVAL, "null argument");
  return run_adjoint(m, k, n_paths, path_offset, seed, 0, d_out, d_paths);
}

}  // extern "C"
