// pc_mlp_tc.cu -- the network's products on the fifth-generation tensor
// cores: tcgen05.mma with the accumulator in tensor memory (TMEM), operands
// staged in shared memory by TMA (cp.async.bulk.tensor) in the 128-byte
// swizzled layouts the MMA reads through its shared-memory descriptors.
//
// C[M, N] = A B^T over K with BF16 operands and FP32 accumulation, in three
// forms (rows = samples, W a layer's weights [out, in]):
//   forward       Z = H W^T      A = H [M][K], B = W [N][K]: both K-major
//   data grad     dH = dZ W      A = dZ [M][K] K-major, B = W [K][N] N-major
//   weight grad   dW = dZ^T H    A = dZ [K][M] M-major, B = H [K][N] N-major,
//                                split over K (the rows) into FP32 partials
// A K-major operand tile is one TMA box of 64 k columns by its rows; an
// MN-major one is BM / 64 (BN / 64) boxes of 64 k rows by 64 columns, the
// MN-major swizzled layout (descriptors sw128_desc / sw128_desc_mn).
//
// The kernel is persistent: one CTA per SM walks the
// output tiles (128 x BN, BN = 64 or 128; with the k splits as a third tile
// coordinate):
//   warp 0, lane 0    TMA producer: 64-deep k chunks into a ring of kStages
//                     stage buffers across tiles, one "full" mbarrier per
//                     stage (expect_tx = the chunk's bytes) and one "empty"
//                     mbarrier the MMA side frees it with;
//   warp 1, lane 0    MMA issuer: four 128 x BN x 16 tcgen05.mma per chunk
//                     into TMEM buffer i & 1 of the CTA's i-th tile (two
//                     buffers of BN columns), tcgen05.commit to the stage's
//                     empty barrier and, after a tile's last chunk, to the
//                     buffer's "tfull" barrier;
//   warps 4..        epilogue, BN / 8 warps (4 + BN / 8 warps in all): warp
//                     w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows) of
//                     columns 32 ((w - 4) / 4) .. + 31 (tcgen05.ld), applies
//                     the product's epilogue (bias + softplus -> BF16; bias ->
//                     FP32; times the softplus derivative from the stored
//                     activation -> BF16; FP32 split partial) and frees the
//                     buffer ("tempty", one arrival per warp), so one tile's
//                     epilogue overlaps the next tile's loads and MMAs.
// Warp 0 allocates 2 BN TMEM columns and frees them once the "done" barrier
// (committed after the last MMA) has completed.  Every wait is bounded
// (about a second of SM clocks) and gives up early once another role has
// given up: on expiry the kernel sets *status, stops issuing work, waits
// (bounded) for its copies and MMAs in flight, frees TMEM and returns; the
// host reports the status.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>

#include "pc_mlp.h"
#include "pc_cv_types.h"

namespace pc {
namespace {

constexpr int kTcBM = 128, kTcBK = 64, kStages = 4, kTcThreads = 384;
constexpr int kEpiWarps = 8;  // warps 4..11 of the table build: two per TMEM lane quarter
// epilogue warps of a product with BN-wide tiles: BN / 32 per TMEM lane
// quarter, each 32 of the tile's columns (8 for BN = 64, 16 for BN = 128)
template <int BN>
__host__ __device__ constexpr int epi_warps() { return BN / 8; }
template <int BN>
__host__ __device__ constexpr int tc_threads() { return 128 + 32 * epi_warps<BN>(); }
constexpr uint32_t kATileBytes = kTcBM * kTcBK * 2;  // 16 KB
constexpr long long kWaitCycles = 2000000000ll;      // ~1 s at 2 GHz
constexpr long long kTestWaitCycles = 20000000ll;    // ~10 ms: the failure test's limit

__device__ __forceinline__ uint32_t su32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of `parity` to complete; false on expiry or
// when *abort is raised (another role of the CTA gave up).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit,
                                          const volatile int *abort = nullptr) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (abort && *abort) return false;
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// layout (rows of 128 bytes, 8-row groups 1024 bytes apart; the group base
// 1024-byte aligned).  Fields: start address >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29, unused by this layout: 1), stride byte offset >> 4
// (32-45: 1024 B), the fixed value 1 at bits 46-48, base offset 0, swizzle
// mode 2 = 128 bytes (61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
         (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B BF16 (7-9 = 1, 10-12 = 1), both K-major (15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn = false, bool b_mn = false) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(a_mn) << 15) | (uint32_t(b_mn) << 16) |
         (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// The same descriptor for an MN-major operand in the 128-byte swizzle
// layout: atoms of 64 M (or N) elements (128 contiguous bytes) by 8 k rows,
// the k rows of an atom 128 bytes apart and the atom's 8-row groups along k
// 1024 bytes apart (stride byte offset), consecutive atoms along M (N)
// kMnAtomBytes apart (leading byte offset: one TMA box of 64 x 64).  A k step
// of 16 is two 8-row groups: the start advances 2048 bytes.
constexpr uint32_t kMnAtomBytes = 64 * 64 * 2;
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(kMnAtomBytes >> 4) << 16) |
         (uint64_t(1024 >> 4) << 32) | (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

__device__ __forceinline__ void mma_bf16_tc(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
  int M, N, K;
  int k_split;                  // k range per blockIdx.z (a multiple of 64)
  const float *bias;
  const __nv_bfloat16 *aux;     // stored activations (kEpiDSoftplus)
  int ldaux;
  __nv_bfloat16 *Cb;
  float *Cf;
  int ldc;
  int splits;                   // k splits (blockIdx-independent: tiles enumerate them)
  int32_t *status;
  // failure test: the producer withholds chunk 0's copies, so the waits on
  // it expire (after wait_cycles) and the kernel takes its abort path
  int withhold;
  long long wait_cycles;
};

// The softplus derivative sigma(z) = 1 - exp(-h) from h = softplus(z) >= 0:
// for h >= 2^-5 with the SFU exponential (absolute error about 1e-7, below
// 4e-6 of the result), below it the series h (1 - h/2 (1 - h/3)) (relative
// error under h^3 / 24 < 2e-6): both far inside the BF16 rounding of dZ.
__device__ __forceinline__ float dsoftplus(float h) {
  return h >= 0.03125f ? 1.f - __expf(-h) : h * fmaf(-0.5f * h, fmaf(-h, 0.3333333333f, 1.f), 1.f);
}

// Output element size of an epilogue (BF16 activations or gradients, FP32
// outputs and partials) and the staging area of one epilogue warp: its 32
// rows by its 32 columns, at most 32 x 32 FP32 values.
template <int EPI>
__host__ __device__ constexpr int out_bytes() { return (EPI == kEpiBiasSoftplus || EPI == kEpiDSoftplus) ? 2 : 4; }
constexpr uint32_t kStageWarpBytes = 32 * 32 * 4;

// The epilogue of 32 accumulator columns of one row (row `row`, columns
// col .. col + 31 of C; bias epilogues add the bias; kEpiDSoftplus reads the
// stored activation), written as 16-byte chunks c0 .. of this lane's row in
// the warp's staging area (rows of rb bytes, chunk c of row r at chunk
// c ^ (r & m), m = min(rb / 16, 8) - 1: the lanes' rows spread over the
// banks, for these writes and for the row-wise copy).
template <int EPI>
__device__ __forceinline__ void epilogue32(const TcArgs &g, int row, int col, const float (&v)[32], uint32_t st,
                                           int lane, int rb, int c0) {
  auto put = [&](int c, uint4 x) {
    const int m = (rb / 16 < 8 ? rb / 16 : 8) - 1;
    const uint32_t a = st + uint32_t(lane * rb + ((c ^ (lane & m)) << 4));
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "r"(x.x), "r"(x.y), "r"(x.z), "r"(x.w)
                 : "memory");
  };
  if (EPI == kEpiBiasSoftplus || EPI == kEpiBias) {
    const float4 *b4 = reinterpret_cast<const float4 *>(g.bias + col);
    float b[32];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 t = __ldg(b4 + q);
      b[4 * q] = t.x; b[4 * q + 1] = t.y; b[4 * q + 2] = t.z; b[4 * q + 3] = t.w;
    }
    if (EPI == kEpiBiasSoftplus) {
      uint32_t pk[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(softplus_fast(v[2 * i] + b[2 * i]),
                                                       softplus_fast(v[2 * i + 1] + b[2 * i + 1]));
        pk[i] = *reinterpret_cast<const uint32_t *>(&h);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) put(c0 + q, make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]));
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        put(c0 + q, make_uint4(__float_as_uint(v[4 * q] + b[4 * q]), __float_as_uint(v[4 * q + 1] + b[4 * q + 1]),
                               __float_as_uint(v[4 * q + 2] + b[4 * q + 2]), __float_as_uint(v[4 * q + 3] + b[4 * q + 3])));
    }
  } else if (EPI == kEpiDSoftplus) {
    // the softplus derivative from the stored activation (32 BF16 values of
    // this row: four 16-byte loads)
    const uint4 *hv = reinterpret_cast<const uint4 *>(g.aux + size_t(row) * g.ldaux + col);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 h4 = __ldg(hv + q);
      const uint32_t hw[4] = {h4.x, h4.y, h4.z, h4.w};
      uint32_t pk[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 hf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hw[e]));
        const int i = 8 * q + 2 * e;
        const __nv_bfloat162 o = __floats2bfloat162_rn(v[i] * dsoftplus(hf.x), v[i + 1] * dsoftplus(hf.y));
        pk[e] = *reinterpret_cast<const uint32_t *>(&o);
      }
      put(c0 + q, make_uint4(pk[0], pk[1], pk[2], pk[3]));
    }
  } else {  // kEpiPartial: this k split's FP32 partial
#pragma unroll
    for (int q = 0; q < 8; ++q)
      put(c0 + q, make_uint4(__float_as_uint(v[4 * q]), __float_as_uint(v[4 * q + 1]), __float_as_uint(v[4 * q + 2]),
                             __float_as_uint(v[4 * q + 3])));
  }
}

// Persistent product: one CTA per SM walks the output tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (tile t: k split t / (tm tn), then row tile,
// then column tile).  The producer streams 64-deep k chunks through a ring
// of kStages stages across tiles; the MMA issuer accumulates tile i into TMEM
// buffer i & 1 (two buffers of BN columns), so the epilogue warps (4..7,
// warp w reading TMEM lanes 32 (w % 4) ..) drain one buffer while the next
// tile's MMAs fill the other.  Barriers: full / empty per stage, tfull /
// tempty per TMEM buffer (tempty: one arrival per epilogue warp), done.
// Warps 2 and 3 have no role (the epilogue warps must sit at positions
// 0..3 of their warp quarter to reach their TMEM lanes).
// AMN / BMN: operand A (B) is M-major (N-major) in memory, loaded as
// BM / 64 (BN / 64) boxes of 64 x 64 in the MN-major swizzled layout.
template <int EPI, int BN, bool AMN, bool BMN>
__global__ void __launch_bounds__(tc_threads<BN>(), 1)
    mlp_gemm_tc(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const TcArgs g) {
  constexpr uint32_t kBTileBytes = BN * kTcBK * 2;
  constexpr uint32_t kStageBytes = kATileBytes + kBTileBytes;
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * kStages + 5];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const volatile int *abort = &abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (g.M + kTcBM - 1) / kTcBM, tn = g.N / BN;
  const int tiles = tm * tn * g.splits;
  const int split_chunks = g.k_split / kTcBK;
  const uint32_t base = (su32(tc_smem_raw) + 1023u) & ~1023u;
  const uint32_t full0 = su32(&bars[0]), empty0 = su32(&bars[kStages]);
  const uint32_t tfull0 = su32(&bars[2 * kStages]), tempty0 = su32(&bars[2 * kStages + 2]);
  const uint32_t done = su32(&bars[2 * kStages + 4]);
  const uint32_t stage0 = base + kStages * kStageBytes;  // epilogue staging, kStageWarpBytes per warp
  auto decode = [&](int t, int &z, int &m0, int &n0, int &c0, int &nk) {
    z = t / (tm * tn);
    const int r = t - z * tm * tn;
    m0 = (r / tn) * kTcBM;
    n0 = (r % tn) * BN;
    c0 = z * split_chunks;
    nk = min(g.k_split, g.K - z * g.k_split) / kTcBK;
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_slot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < 2 * kStages; ++s) mbar_init(su32(&bars[s]), 1);
    mbar_init(tfull0, 1);
    mbar_init(tfull0 + 8, 1);
    mbar_init(tempty0, epi_warps<BN>());
    mbar_init(tempty0 + 8, epi_warps<BN>());
    mbar_init(done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (threadIdx.x == 0) {
    // TMA producer: chunk counter q runs across this CTA's tiles
    uint32_t q = 0, issued = 0;  // chunks issued: their copies land before exit
    for (int t = blockIdx.x; t < tiles && !*abort; t += gridDim.x) {
      int z, m0, n0, c0, nk;
      decode(t, z, m0, n0, c0, nk);
      for (int c = 0; c < nk; ++c, ++q) {
        const uint32_t s = q % kStages, u = q / kStages;
        if (u >= 1 && !mbar_wait(empty0 + 8 * s, (u - 1) & 1, g.wait_cycles, abort)) {
          if (!*abort) atomicOr(g.status, 4);
          atomicExch(&abort_flag, 1);
          break;
        }
        if (g.withhold && q == 0) continue;  // failure test: chunk 0 never arrives
        const uint32_t sa = base + s * kStageBytes, sb = sa + kATileBytes;
        const int kc = (c0 + c) * kTcBK;
        mbar_expect_tx(full0 + 8 * s, kStageBytes);
        if (AMN) {
#pragma unroll
          for (int b = 0; b < kTcBM / 64; ++b) tma_load_2d(sa + b * kMnAtomBytes, &ta, m0 + 64 * b, kc, full0 + 8 * s);
        } else {
          tma_load_2d(sa, &ta, kc, m0, full0 + 8 * s);
        }
        if (BMN) {
#pragma unroll
          for (int b = 0; b < BN / 64; ++b) tma_load_2d(sb + b * kMnAtomBytes, &tb, n0 + 64 * b, kc, full0 + 8 * s);
        } else {
          tma_load_2d(sb, &tb, kc, n0, full0 + 8 * s);
        }
        issued = q + 1;
      }
    }
    // the last kStages issued chunks' copies complete before the CTA exits
    for (uint32_t c = issued > kStages ? issued - kStages : 0; c < issued; ++c)
      if (!(g.withhold && c == 0) && !mbar_wait(full0 + 8 * (c % kStages), (c / kStages) & 1, g.wait_cycles))
        atomicOr(g.status, 4);
  } else if (threadIdx.x == 32) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(kTcBM, BN, AMN, BMN);
    uint32_t q = 0;
    int i = 0;
    for (int t = blockIdx.x; t < tiles && !*abort; t += gridDim.x, ++i) {
      int z, m0, n0, c0, nk;
      decode(t, z, m0, n0, c0, nk);
      const int buf = i & 1, v = i >> 1;
      if (v >= 1 && !mbar_wait(tempty0 + 8 * buf, (v - 1) & 1, g.wait_cycles, abort)) {
        if (!*abort) atomicOr(g.status, 4);
        atomicExch(&abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t acc = tmem + uint32_t(buf * BN);
      bool ok = true;
      for (int c = 0; c < nk; ++c, ++q) {
        const uint32_t s = q % kStages, u = q / kStages;
        if (!mbar_wait(full0 + 8 * s, u & 1, g.wait_cycles, abort)) {
          if (!*abort) atomicOr(g.status, 4);
          atomicExch(&abort_flag, 1);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t sa = base + s * kStageBytes, sb = sa + kATileBytes;
#pragma unroll
        for (int kk = 0; kk < kTcBK / 16; ++kk) {
          const uint64_t da = AMN ? sw128_desc_mn(sa + kk * 2048) : sw128_desc(sa + kk * 32);
          const uint64_t db = BMN ? sw128_desc_mn(sb + kk * 2048) : sw128_desc(sb + kk * 32);
          mma_bf16_tc(acc, da, db, idesc, (c | kk) != 0);
        }
        mma_commit(empty0 + 8 * s);
      }
      if (!ok) break;
      mma_commit(tfull0 + 8 * buf);
    }
    // every MMA this thread issued completes before `done`
    mma_commit(done);
  } else if (warp >= 4) {
    // epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31 (rows of the
    // tile), columns 32 ((w - 4) / 4) .. + 31 of it
    const int qw = warp & 3, grp = (warp - 4) >> 2;
    int i = 0;
    for (int t = blockIdx.x; t < tiles && !*abort; t += gridDim.x, ++i) {
      int z, m0, n0, c0, nk;
      decode(t, z, m0, n0, c0, nk);
      const int buf = i & 1, v = i >> 1;
      if (!mbar_wait(tfull0 + 8 * buf, v & 1, g.wait_cycles, abort)) {
        if (!*abort) atomicOr(g.status, 4);
        atomicExch(&abort_flag, 1);
        break;
      }
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int row = m0 + 32 * qw + lane;
      const uint32_t trow = tmem + (uint32_t(32 * qw) << 16) + uint32_t(buf * BN);
      // this warp's 32 rows x 32 columns, staged as rows of rb bytes
      constexpr int EB = out_bytes<EPI>();
      constexpr int rb = 32 * EB;
      const uint32_t st = stage0 + uint32_t(warp - 4) * kStageWarpBytes;
      const int col0 = n0 + grp * 32;
#pragma unroll 1
      for (int j = 0; j < 32; j += 32) {
        float r[32];
        tmem_ld32(trow + grp * 32 + j, r);
        if (row < g.M) epilogue32<EPI>(g, row, col0 + j, r, st, lane, rb, j * EB / 16);
      }
      // the accumulator buffer is free once read
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
      // row-wise copy to C: CPR lanes per row, each 16 bytes (whole lines)
      {
        constexpr int CPR = rb / 16, RPI = 32 / CPR, SW = (CPR < 8 ? CPR : 8) - 1;
        const int rr = lane / CPR, cc = lane % CPR;
        char *cbase = EPI == kEpiBiasSoftplus || EPI == kEpiDSoftplus
                          ? reinterpret_cast<char *>(g.Cb)
                          : reinterpret_cast<char *>(g.Cf + (EPI == kEpiPartial ? size_t(z) * size_t(g.M) * g.ldc : 0));
#pragma unroll 4
        for (int r0 = 0; r0 < 32; r0 += RPI) {
          const int lr = r0 + rr, grow = m0 + 32 * qw + lr;
          uint4 x;
          const uint32_t a = st + uint32_t(lr * rb + ((cc ^ (lr & SW)) << 4));
          asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];\n"
                       : "=r"(x.x), "=r"(x.y), "=r"(x.z), "=r"(x.w)
                       : "r"(a)
                       : "memory");
          if (grow < g.M)
            *reinterpret_cast<uint4 *>(cbase + (size_t(grow) * g.ldc + col0) * EB + size_t(cc) * 16) = x;
        }
        __syncwarp();
      }
    }
  }
  __syncwarp();
  // every MMA has completed before TMEM is released
  if (warp == 0 && !mbar_wait(done, 0, g.wait_cycles)) atomicOr(g.status, 4);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * BN));
  }
}

// ---------------------------------------------------------------------------
// The hedge tables in one launch (cv_tables_tc): one CTA per 128-row tile
// (persistent over tiles), the tile's activations resident in shared memory
// between layers.  Shared memory: A, the current layer's input, 128 rows x
// up to 256 columns as four K-major 128-byte-swizzled blocks of 64 columns
// (16 KB each, what the MMA's A descriptor reads); a ring of kStages weight
// stages of up to 256 rows x 64 k (32 KB, written by TMA).  Roles:
//   thread 0      TMA producer: every layer's 64-deep weight chunks, in
//                 order, through the ring (full / empty barriers);
//   thread 32     MMA issuer: per layer, once its input is in A ("aready",
//                 one arrival per epilogue warp), wp[l] / 64 chunks of four
//                 128 x N x 16 tcgen05.mma into TMEM columns 0 .. N - 1, then
//                 a commit to "afull";
//   warps 4..11   epilogue: the tile's inputs (features) into A block 0;
//                 after each hidden layer's "afull", bias + softplus of their
//                 32 rows x N / 2 columns back into A as BF16 (the next
//                 layer's input); after the last layer, the hedge ratios to
//                 the tables.  A and TMEM are single buffers: a layer's MMAs
//                 start only after the epilogue has read TMEM and written A,
//                 and the epilogue writes A only after the MMAs reading it
//                 completed.
constexpr uint32_t kFzABytes = 4 * kATileBytes;       // 64 KB
constexpr uint32_t kFzStageBytes = 256 * kTcBK * 2;   // 32 KB
constexpr size_t kFzSmem = 1024 + size_t(kFzABytes) + size_t(kStages) * kFzStageBytes;

__device__ __forceinline__ void st_shared16(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}
// 16-byte chunk ch (of 8) of row r in a K-major 128-byte-swizzled block
__device__ __forceinline__ uint32_t sw128_chunk(uint32_t block, int r, int ch) {
  return block + uint32_t(r * 128 + ((ch ^ (r & 7)) << 4));
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}
// generic-proxy writes to shared memory visible to the tensor core's reads
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1)
    cv_tables_tc(const __grid_constant__ CvTablesTc t, const __grid_constant__ CvArgs c,
                 const __grid_constant__ CvFeatureArgs fa) {
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * kStages + 3];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const volatile int *abort = &abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = int((t.rows + kTcBM - 1) / kTcBM);
  const uint32_t abuf = (su32(tc_smem_raw) + 1023u) & ~1023u, ring = abuf + kFzABytes;
  const uint32_t full0 = su32(&bars[0]), empty0 = su32(&bars[kStages]);
  const uint32_t aready = su32(&bars[2 * kStages]), afull = aready + 8, done = aready + 16;
  const long long lim = t.withhold ? kTestWaitCycles : kWaitCycles;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_slot)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < 2 * kStages; ++s) mbar_init(su32(&bars[s]), 1);
    mbar_init(aready, kEpiWarps);
    mbar_init(afull, 1);
    mbar_init(done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (threadIdx.x == 0) {
    // TMA producer: chunk counter q runs across layers and tiles
    uint32_t q = 0, issued = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < tiles && ok && !*abort; tile += gridDim.x) {
      for (int l = 0; l < t.L && ok; ++l) {
        const int nk = t.wp[l] / kTcBK;
        const uint32_t bytes = uint32_t(t.wp[l + 1]) * kTcBK * 2;
        for (int ch = 0; ch < nk; ++ch, ++q) {
          const uint32_t s = q % kStages, u = q / kStages;
          if (u >= 1 && !mbar_wait(empty0 + 8 * s, (u - 1) & 1, lim, abort)) {
            if (!*abort) atomicOr(t.status, 4);
            atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
          issued = q + 1;
          if (t.withhold && q == 0) continue;  // failure test: chunk 0 never arrives
          mbar_expect_tx(full0 + 8 * s, bytes);
          tma_load_2d(ring + s * kFzStageBytes, &t.w[l], ch * kTcBK, 0, full0 + 8 * s);
        }
      }
    }
    // the last kStages issued chunks' copies complete before the CTA exits
    for (uint32_t k = issued > kStages ? issued - kStages : 0; k < issued; ++k)
      if (!(t.withhold && k == 0) && !mbar_wait(full0 + 8 * (k % kStages), (k / kStages) & 1, lim))
        atomicOr(t.status, 4);
  } else if (threadIdx.x == 32) {
    // MMA issuer; ph counts the layers issued (the aready / afull phases)
    uint32_t q = 0, ph = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < tiles && ok && !*abort; tile += gridDim.x) {
      for (int l = 0; l < t.L && ok; ++l, ++ph) {
        if (!mbar_wait(aready, ph & 1, lim, abort)) {
          if (!*abort) atomicOr(t.status, 4);
          atomicExch(&abort_flag, 1);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t idesc = idesc_bf16(kTcBM, t.wp[l + 1]);
        const int nk = t.wp[l] / kTcBK;
        for (int ch = 0; ch < nk; ++ch, ++q) {
          const uint32_t s = q % kStages, u = q / kStages;
          if (!mbar_wait(full0 + 8 * s, u & 1, lim, abort)) {
            if (!*abort) atomicOr(t.status, 4);
            atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t sa = abuf + uint32_t(ch) * kATileBytes, sb = ring + s * kFzStageBytes;
#pragma unroll
          for (int kk = 0; kk < kTcBK / 16; ++kk)
            mma_bf16_tc(tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), idesc, (ch | kk) != 0);
          mma_commit(empty0 + 8 * s);
        }
        if (ok) mma_commit(afull);
      }
    }
    // every MMA this thread issued completes before `done`
    mma_commit(done);
  } else if (warp >= 4) {
    // epilogue: warp w owns TMEM lanes (tile rows) 32 (w % 4) .. + 31 and
    // half (w - 4) / 4 of each layer's columns; ph counts the layers drained
    const int qw = warp & 3, half = (warp - 4) >> 2, rl = 32 * qw + lane;
    const uint32_t trow = tmem + (uint32_t(32 * qw) << 16);
    uint32_t ph = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < tiles && ok && !*abort; tile += gridDim.x) {
      const size_t r = size_t(tile) * kTcBM + size_t(rl);
      // layer 0's input: the row's 16 features (columns 0..15 of block 0),
      // zeros up to column 63
      if (half == 0) {
        float f[kCvFeatures];
        if (r < t.rows) {
          cv_feature_row(c, fa, r, t.rows, f);
        } else {
#pragma unroll
          for (int i = 0; i < kCvFeatures; ++i) f[i] = 0.f;
        }
        uint32_t pk[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) pk[i] = pack_bf16(f[2 * i], f[2 * i + 1]);
        st_shared16(sw128_chunk(abuf, rl, 0), pk[0], pk[1], pk[2], pk[3]);
        st_shared16(sw128_chunk(abuf, rl, 1), pk[4], pk[5], pk[6], pk[7]);
        st_shared16(sw128_chunk(abuf, rl, 2), 0u, 0u, 0u, 0u);
        st_shared16(sw128_chunk(abuf, rl, 3), 0u, 0u, 0u, 0u);
      } else {
#pragma unroll
        for (int ch = 4; ch < 8; ++ch) st_shared16(sw128_chunk(abuf, rl, ch), 0u, 0u, 0u, 0u);
      }
      fence_async_shared();
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(aready);
      for (int l = 0; l < t.L; ++l, ++ph) {
        if (!mbar_wait(afull, ph & 1, lim, abort)) {
          if (!*abort) atomicOr(t.status, 4);
          atomicExch(&abort_flag, 1);
          ok = false;
          break;
        }
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (l + 1 < t.L) {
          // bias + softplus -> BF16 into A, the next layer's input
          const int cols = t.wp[l + 1] / 2, c0 = half * cols;
#pragma unroll 1
          for (int j = 0; j < cols; j += 32) {
            const int col = c0 + j;
            float v[32];
            tmem_ld32(trow + uint32_t(col), v);
            const float4 *b4 = reinterpret_cast<const float4 *>(t.bias[l] + col);
            uint32_t pk[16];
#pragma unroll
            for (int q4 = 0; q4 < 8; ++q4) {
              const float4 b = __ldg(b4 + q4);
              pk[2 * q4] = pack_bf16(softplus_fast(v[4 * q4] + b.x), softplus_fast(v[4 * q4 + 1] + b.y));
              pk[2 * q4 + 1] = pack_bf16(softplus_fast(v[4 * q4 + 2] + b.z), softplus_fast(v[4 * q4 + 3] + b.w));
            }
            const uint32_t blk = abuf + uint32_t(col >> 6) * kATileBytes;
            const int ch0 = (col & 63) >> 3;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4)
              st_shared16(sw128_chunk(blk, rl, ch0 + q4), pk[4 * q4], pk[4 * q4 + 1], pk[4 * q4 + 2], pk[4 * q4 + 3]);
          }
          fence_async_shared();
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(aready);
        } else if (half == 0) {
          // the last layer: hedge ratios (outputs 1 .. d) + bias
          float v[32];
          tmem_ld32(trow, v);
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
          if (r < t.rows) {
#pragma unroll
            for (int i = 0; i < kCvMaxD; ++i) {
              if (i >= c.d) break;
              const float y = v[1 + i] + __ldg(t.bias[l] + 1 + i);
              if (r + 1 < t.rows) t.tables[r * kCvRecord + i] = y;
              else t.delta0[i] = y;
            }
          }
        }
      }
    }
  }
  __syncwarp();
  // every MMA has completed before TMEM is released
  if (warp == 0 && !mbar_wait(done, 0, lim)) atomicOr(t.status, 4);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(256));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2-D BF16 tensor [rows, cols] (cols contiguous, row stride ld elements),
// box of box_rows x box_cols, 128-byte swizzle, zero fill out of range.
bool make_map(CUtensorMap &m, const __nv_bfloat16 *p, uint64_t rows, uint64_t cols, uint64_t ld,
              uint32_t box_rows, uint32_t box_cols = kTcBK) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {ld * 2};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(p), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
constexpr size_t tc_smem() {
  return size_t(kStages) * (kATileBytes + size_t(BN) * kTcBK * 2) + size_t(epi_warps<BN>()) * kStageWarpBytes + 1024;
}

int sm_count() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 1;
  });
  return n;
}

// Persistent grid: the tiles, at most one CTA per SM.
template <int EPI, int BN, bool AMN, bool BMN>
cudaError_t launch_tc(const CUtensorMap &ta, const CUtensorMap &tb, const TcArgs &a, cudaStream_t s) {
  const long long tiles = (long long)(a.N / BN) * ((a.M + kTcBM - 1) / kTcBM) * a.splits;
  const long long cap = (long long)sm_count();
  const unsigned grid = unsigned(tiles < cap ? tiles : cap);
  mlp_gemm_tc<EPI, BN, AMN, BMN><<<grid, tc_threads<BN>(), tc_smem<BN>(), s>>>(ta, tb, a);
  return cudaGetLastError();
}

template <int EPI, bool AMN, bool BMN>
cudaError_t tc_attr() {
  cudaError_t r = cudaFuncSetAttribute(mlp_gemm_tc<EPI, 64, AMN, BMN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(tc_smem<64>()));
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(mlp_gemm_tc<EPI, 128, AMN, BMN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(tc_smem<128>()));
  return r;
}

}  // namespace

cudaError_t gemm_tc_init() {
  static std::once_flag once;
  static cudaError_t r = cudaSuccess;
  std::call_once(once, [] {
    int dev = 0, major = 0;
    r = cudaGetDevice(&dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (r == cudaSuccess && major < 10) r = cudaErrorNotSupported;
    if (r == cudaSuccess && !encode_fn()) r = cudaErrorNotSupported;
    if (r == cudaSuccess) r = tc_attr<kEpiBiasSoftplus, false, false>();
    if (r == cudaSuccess) r = tc_attr<kEpiBias, false, false>();
    if (r == cudaSuccess) r = tc_attr<kEpiDSoftplus, false, true>();
    if (r == cudaSuccess) r = tc_attr<kEpiPartial, true, true>();
  });
  return r;
}

bool gemm_tc_supported(GemmKind kind, const GemmArgs &g) {
  const bool shape = g.K % kTcBK == 0 && g.K >= kTcBK && g.M % 64 == 0 && g.M > 0 &&
                     (g.N == 64 || g.N % 128 == 0) && g.lda % 8 == 0 && g.ldb % 8 == 0 && g.ldc % 8 == 0;
  if (!shape) return false;
  if (kind == kGemmDataGrad) return g.aux != nullptr && g.ldaux % 8 == 0;
  if (kind == kGemmWeightGrad) return g.k_split % kTcBK == 0 && g.k_split > 0;
  return true;
}

bool make_tc_maps(GemmKind kind, const GemmArgs &g, TcMaps &m) {
  if (!gemm_tc_supported(kind, g) || gemm_tc_init() != cudaSuccess) return false;
  const uint32_t bn = g.N == 64 ? 64 : 128;
  switch (kind) {
    case kGemmForward:  // A [M][K], B [N][K]
      return make_map(m.a, g.A, uint64_t(g.M), uint64_t(g.K), uint64_t(g.lda), kTcBM) &&
             make_map(m.b, g.B, uint64_t(g.N), uint64_t(g.K), uint64_t(g.ldb), bn);
    case kGemmDataGrad:  // A [M][K], B [K][N] (N-major: boxes of 64 k rows x 64 columns)
      return make_map(m.a, g.A, uint64_t(g.M), uint64_t(g.K), uint64_t(g.lda), kTcBM) &&
             make_map(m.b, g.B, uint64_t(g.K), uint64_t(g.N), uint64_t(g.ldb), kTcBK, 64);
    case kGemmWeightGrad:  // A [K][M] (M-major), B [K][N] (N-major)
      return make_map(m.a, g.A, uint64_t(g.K), uint64_t(g.M), uint64_t(g.lda), kTcBK, 64) &&
             make_map(m.b, g.B, uint64_t(g.K), uint64_t(g.N), uint64_t(g.ldb), kTcBK, 64);
  }
  return false;
}

cudaError_t launch_gemm_tc(GemmKind kind, int epi, const GemmArgs &g, const TcMaps &m, int splits,
                           int32_t *status, cudaStream_t s, bool withhold) {
  if (!status || !gemm_tc_supported(kind, g)) return cudaErrorInvalidValue;
  const bool ok_epi = kind == kGemmForward ? (epi == kEpiBiasSoftplus || epi == kEpiBias)
                      : kind == kGemmDataGrad ? epi == kEpiDSoftplus
                                              : epi == kEpiPartial;
  if (!ok_epi) return cudaErrorInvalidValue;
  // every split has at least one k chunk
  const int k_split = kind == kGemmWeightGrad ? g.k_split : g.K;
  if (splits < 1 || (kind != kGemmWeightGrad && splits != 1) || (splits - 1) * k_split >= g.K ||
      splits * k_split < g.K)
    return cudaErrorInvalidValue;
  const cudaError_t r = gemm_tc_init();
  if (r != cudaSuccess) return r;
  TcArgs a{};
  a.M = g.M;
  a.N = g.N;
  a.K = g.K;
  a.k_split = k_split;
  a.splits = splits;
  a.bias = g.bias;
  a.aux = g.aux;
  a.ldaux = g.ldaux;
  a.Cb = g.Cb;
  a.Cf = g.Cf;
  a.ldc = g.ldc;
  a.status = status;
  a.withhold = withhold ? 1 : 0;
  a.wait_cycles = withhold ? kTestWaitCycles : kWaitCycles;
  const bool n64 = g.N == 64;
  switch (kind) {
    case kGemmForward:
      if (epi == kEpiBiasSoftplus)
        return n64 ? launch_tc<kEpiBiasSoftplus, 64, false, false>(m.a, m.b, a, s)
                   : launch_tc<kEpiBiasSoftplus, 128, false, false>(m.a, m.b, a, s);
      return n64 ? launch_tc<kEpiBias, 64, false, false>(m.a, m.b, a, s)
                 : launch_tc<kEpiBias, 128, false, false>(m.a, m.b, a, s);
    case kGemmDataGrad:
      return n64 ? launch_tc<kEpiDSoftplus, 64, false, true>(m.a, m.b, a, s)
                 : launch_tc<kEpiDSoftplus, 128, false, true>(m.a, m.b, a, s);
    case kGemmWeightGrad:
      return n64 ? launch_tc<kEpiPartial, 64, true, true>(m.a, m.b, a, s)
                 : launch_tc<kEpiPartial, 128, true, true>(m.a, m.b, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pc

namespace pc {

bool cv_tables_tc_shape(int L, const int *wp) {
  if (L < 2 || L > kCvNetMaxLayers || wp[0] != kTcBK || wp[L] != kTcBK) return false;
  for (int l = 1; l < L; ++l)
    if (wp[l] % kTcBK || wp[l] > 256) return false;
  return true;
}

bool make_weight_map(CUtensorMap &m, const __nv_bfloat16 *w, int n_out, int n_in) {
  if (gemm_tc_init() != cudaSuccess || n_out > 256) return false;
  return make_map(m, w, uint64_t(n_out), uint64_t(n_in), uint64_t(n_in), uint32_t(n_out));
}

cudaError_t launch_cv_tables_tc(const CvTablesTc &t, const CvArgs &c, const CvFeatureArgs &fa, cudaStream_t s) {
  if (!t.status || !t.tables || !t.delta0 || t.rows < 1 || !cv_tables_tc_shape(t.L, t.wp))
    return cudaErrorInvalidValue;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = gemm_tc_init();
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(cv_tables_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kFzSmem));
  });
  if (attr != cudaSuccess) return attr;
  const long long tiles = (long long)((t.rows + kTcBM - 1) / kTcBM), cap = (long long)sm_count();
  cv_tables_tc<<<unsigned(tiles < cap ? tiles : cap), kTcThreads, kFzSmem, s>>>(t, c, fa);
  return cudaGetLastError();
}

}  // namespace pc
