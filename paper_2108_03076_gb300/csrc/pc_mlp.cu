// pc_mlp.cu -- the learned control variate's network on the tensor cores:
// a BF16 multilayer perceptron with FP32 accumulation (forward, backward,
// Adam), and the kernels that turn it into hedge-ratio tables.
//
// Every matrix product is one kernel, mlp_gemm: 64x64 output tiles, 32-deep
// k steps staged in shared memory by cp.async (two stages), fragments read
// with ldmatrix (.trans for operands stored M- or N-major) and multiplied
// with mma.sync m16n8k16 BF16 -> FP32.  Samples are rows: activations are
// [rows, features] BF16, weights [out, in] row-major BF16 copies of FP32
// master weights.  The three products of a layer are
//   forward      Z = H W^T      (A = H, K-major;   B = W,  K-major)
//   data grad    dH = dZ W      (A = dZ, K-major;  B = W,  N-major)
//   weight grad  dW = dZ^T H    (A = dZ, M-major;  B = H,  N-major),
// the last split over the batch (k) into partials summed in a fixed order,
// so every result is deterministic.  Epilogues fuse the bias and softplus
// (forward), the softplus derivative sigma(z) = 1 - exp(-softplus(z)) read
// back from the stored activation (data grad), or write FP32 partials.
#include <cuda_bf16.h>
#include <cstdint>

#include "pc_device.cuh"
#include "pc_mlp.h"

namespace pc {
namespace {

constexpr int BM = 64, BN = 64, BK = 32;
constexpr int SK = BK + 8;   // K-major tile row stride (halves): 80 B rows
constexpr int SC = BM + 8;   // M/N-major tile row stride (halves): 144 B rows
constexpr int kTileHalves = (BM * SK > BK * SC ? BM * SK : BK * SC);

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage one k step of an operand: a K-major operand tile is 64 rows of 32
// halves (row r at s + r*SK), an M/N-major one 32 rows (k) of 64 halves
// (row k at s + k*SC).  128 threads, two 16-byte chunks each.
template <bool KMAJOR>
__device__ __forceinline__ void stage(__nv_bfloat16 *s, const __nv_bfloat16 *g, int ld, int row0, int k0) {
#pragma unroll
  for (int c = threadIdx.x; c < 256; c += 128) {
    if (KMAJOR) {
      const int r = c >> 2, col = (c & 3) * 8;
      cp_async16(s + r * SK + col, g + size_t(row0 + r) * ld + k0 + col);
    } else {
      const int k = c >> 3, col = (c & 7) * 8;
      cp_async16(s + k * SC + col, g + size_t(k0 + k) * ld + row0 + col);
    }
  }
}

template <bool A_KM, bool B_KM, int EPI>
__global__ void __launch_bounds__(128) mlp_gemm(const GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 sA[2][kTileHalves];
  __shared__ __align__(16) __nv_bfloat16 sB[2][kTileHalves];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * g.k_split, ke = min(g.K, kb + g.k_split);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[i][j][v] = 0.f;
  const int steps = (ke - kb) / BK;
  if (steps > 0) {
    stage<A_KM>(sA[0], g.A, g.lda, m0, kb);
    stage<B_KM>(sB[0], g.B, g.ldb, n0, kb);
    cp_async_commit();
  }
  for (int s = 0; s < steps; ++s) {
    const int cur = s & 1;
    if (s + 1 < steps) {
      stage<A_KM>(sA[cur ^ 1], g.A, g.lda, m0, kb + (s + 1) * BK);
      stage<B_KM>(sB[cur ^ 1], g.B, g.ldb, n0, kb + (s + 1) * BK);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const __nv_bfloat16 *a = sA[cur], *b = sB[cur];
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bf[2][4];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int mb = wm * 32 + mi * 16;
        if (A_KM)
          ldsm_x4(af[mi], a + (mb + (lane & 15)) * SK + ks + (lane >> 4) * 8);
        else
          ldsm_x4_t(af[mi], a + (ks + (lane & 7) + (lane >> 4) * 8) * SC + mb + ((lane >> 3) & 1) * 8);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int nb = wn * 32 + np * 16;
        if (B_KM)
          ldsm_x4(bf[np], b + (nb + (lane & 7) + (lane >> 4) * 8) * SK + ks + ((lane >> 3) & 1) * 8);
        else
          ldsm_x4_t(bf[np], b + (ks + (lane & 7) + ((lane >> 3) & 1) * 8) * SC + nb + (lane >> 4) * 8);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          mma_bf16(acc[mi][ni], af[mi], bf[ni >> 1][(ni & 1) * 2], bf[ni >> 1][(ni & 1) * 2 + 1]);
    }
    __syncthreads();
  }
  // epilogue: thread holds rows r, r + 8 and columns c, c + 1 of each 16x8 tile
#pragma unroll
  for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const int c = n0 + wn * 32 + ni * 8 + (lane & 3) * 2;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = m0 + wm * 32 + mi * 16 + (lane >> 2) + h * 8;
        float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
        if (EPI == kEpiBiasSoftplus || EPI == kEpiBias) {
          v0 += g.bias[c];
          v1 += g.bias[c + 1];
        }
        if (EPI == kEpiBiasSoftplus) {
          *reinterpret_cast<__nv_bfloat162 *>(g.Cb + size_t(r) * g.ldc + c) =
              __floats2bfloat162_rn(softplus_fast(v0), softplus_fast(v1));
        } else if (EPI == kEpiBias) {
          *reinterpret_cast<float2 *>(g.Cf + size_t(r) * g.ldc + c) = make_float2(v0, v1);
        } else if (EPI == kEpiDSoftplus) {
          const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162 *>(g.aux + size_t(r) * g.ldaux + c);
          const float2 hf = __bfloat1622float2(hv);
          v0 *= -expm1f(-hf.x);
          v1 *= -expm1f(-hf.y);
          *reinterpret_cast<__nv_bfloat162 *>(g.Cb + size_t(r) * g.ldc + c) = __floats2bfloat162_rn(v0, v1);
        } else {  // kEpiPartial
          float *out = g.Cf + size_t(blockIdx.z) * size_t(g.M) * g.ldc;
          *reinterpret_cast<float2 *>(out + size_t(r) * g.ldc + c) = make_float2(v0, v1);
        }
      }
    }
  }
}

}  // namespace

namespace {

__global__ void to_bf16_kernel(const float *x, size_t n, int fin, __nv_bfloat16 *X, size_t rows, int ld) {
  const size_t total = rows * size_t(ld);
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < total; e += size_t(gridDim.x) * blockDim.x) {
    const size_t r = e / ld;
    const int c = int(e % ld);
    X[e] = __float2bfloat16_rn(r < n && c < fin ? x[r * fin + c] : 0.f);
  }
}

__global__ void gather_kernel(const float *x, const float *t, size_t n_data, int fin, int fout,
                              const uint64_t *step, uint32_t s0, uint32_t s1, size_t batch,
                              __nv_bfloat16 *X, int ldx, float *T) {
  const size_t b = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (b >= batch) return;
  const uint64_t st = *step;
  // the first word of Philox4x32-10 at counter (b, step), key (s0, s1)
  const uint32_t u = philox(make_uint4(uint32_t(b), uint32_t(b >> 32), uint32_t(st), uint32_t(st >> 32)), s0, s1).x;
  const size_t src = size_t(u) % n_data;
  for (int c = 0; c < ldx; ++c) X[b * ldx + c] = __float2bfloat16_rn(c < fin ? x[src * fin + c] : 0.f);
  for (int c = 0; c < fout; ++c) T[b * fout + c] = t[src * fout + c];
}

__global__ void loss_kernel(const float *Y, int ldy, const float *T, const float *w, size_t n, int fout,
                            size_t rows, __nv_bfloat16 *dY, int ldd, float *part) {
  __shared__ float red[32];
  const size_t total = rows * size_t(ldd);
  float acc = 0.f;
  const float inv = 1.f / float(n);
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < total; e += size_t(gridDim.x) * blockDim.x) {
    const size_t r = e / ldd;
    const int c = int(e % ldd);
    float g = 0.f;
    if (r < n && c < fout) {
      const float diff = Y[r * ldy + c] - T[r * fout + c];
      acc += w[c] * diff * diff * inv;
      g = 2.f * w[c] * diff * inv;
    }
    dY[e] = __float2bfloat16_rn(g);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) s += red[i];
    part[blockIdx.x] = s;
  }
}

__global__ void split_sum_kernel(const float *part, int splits, size_t stride, size_t count, float *out) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < count; i += size_t(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[size_t(z) * stride + i];
    out[i] = s;
  }
}

constexpr int kColChunk = 256;

__global__ void colsum_kernel(const __nv_bfloat16 *dZ, size_t rows, int ld, int cols, float *scratch) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const size_t r0 = size_t(blockIdx.y) * kColChunk, r1 = min(rows, r0 + kColChunk);
  float s = 0.f;
  for (size_t r = r0; r < r1; ++r) s += __bfloat162float(dZ[r * ld + c]);
  scratch[size_t(blockIdx.y) * cols + c] = s;
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, size_t n,
                            const uint64_t *step, float lr, float b1, float b2, float eps) {
  const double t = double(*step + 1);
  const float c1 = float(1.0 - pow(double(b1), t)), c2 = float(1.0 - pow(double(b2), t));
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void loss_total_kernel(const float *part, int blocks, double *loss, uint64_t *step) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < blocks; ++i) s += double(part[i]);
  *loss = s;
  if (step) *step += 1;
}

__global__ void unpad_kernel(const float *Y, int ldy, size_t n, int fout, float *y) {
  const size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (e >= n * size_t(fout)) return;
  y[e] = Y[(e / fout) * ldy + e % fout];
}

unsigned grid_for(size_t work, int block, unsigned cap = 4096) {
  size_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  return unsigned(g < cap ? g : cap);
}

}  // namespace

cudaError_t launch_gemm(GemmKind kind, int epi, const GemmArgs &g, int splits, cudaStream_t s) {
  if (g.M % BM || g.N % BN || g.K % BK || g.k_split % BK || splits < 1) return cudaErrorInvalidValue;
  const dim3 grid(unsigned(g.N / BN), unsigned(g.M / BM), unsigned(splits));
  switch (kind) {
    case kGemmForward:
      if (epi == kEpiBiasSoftplus) mlp_gemm<true, true, kEpiBiasSoftplus><<<grid, 128, 0, s>>>(g);
      else if (epi == kEpiBias) mlp_gemm<true, true, kEpiBias><<<grid, 128, 0, s>>>(g);
      else return cudaErrorInvalidValue;
      break;
    case kGemmDataGrad:
      if (epi != kEpiDSoftplus) return cudaErrorInvalidValue;
      mlp_gemm<true, false, kEpiDSoftplus><<<grid, 128, 0, s>>>(g);
      break;
    case kGemmWeightGrad:
      if (epi != kEpiPartial) return cudaErrorInvalidValue;
      mlp_gemm<false, false, kEpiPartial><<<grid, 128, 0, s>>>(g);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *x, size_t n, int fin, __nv_bfloat16 *X, size_t rows, int ld,
                           cudaStream_t s) {
  to_bf16_kernel<<<grid_for(rows * ld, 256), 256, 0, s>>>(x, n, fin, X, rows, ld);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float *x, const float *t, size_t n_data, int fin, int fout,
                          const uint64_t *step, uint32_t s0, uint32_t s1, size_t batch,
                          __nv_bfloat16 *X, int ldx, float *T, cudaStream_t s) {
  gather_kernel<<<unsigned((batch + 127) / 128), 128, 0, s>>>(x, t, n_data, fin, fout, step, s0, s1, batch,
                                                              X, ldx, T);
  return cudaGetLastError();
}

int loss_blocks(size_t rows) { return int(grid_for(rows * 64, 256, 512)); }

cudaError_t launch_loss(const float *Y, int ldy, const float *T, const float *w, size_t n, int fout,
                        size_t rows, __nv_bfloat16 *dY, int ldd, float *part, int blocks, cudaStream_t s) {
  loss_kernel<<<blocks, 256, 0, s>>>(Y, ldy, T, w, n, fout, rows, dY, ldd, part);
  return cudaGetLastError();
}

cudaError_t launch_split_sum(const float *part, int splits, size_t stride, size_t count, float *out,
                             cudaStream_t s) {
  split_sum_kernel<<<grid_for(count, 256), 256, 0, s>>>(part, splits, stride, count, out);
  return cudaGetLastError();
}

cudaError_t launch_colsum(const __nv_bfloat16 *dZ, size_t rows, int ld, int cols, float *scratch,
                          float *out, cudaStream_t s) {
  const unsigned chunks = unsigned((rows + kColChunk - 1) / kColChunk);
  colsum_kernel<<<dim3(unsigned((cols + 127) / 128), chunks), 128, 0, s>>>(dZ, rows, ld, cols, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_split_sum(scratch, int(chunks), size_t(cols), size_t(cols), out, s);
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, size_t n,
                        uint64_t *step, float lr, float b1, float b2, float eps, cudaStream_t s) {
  adam_kernel<<<grid_for(n, 256, 1024), 256, 0, s>>>(p, g, m, v, pb, n, step, lr, b1, b2, eps);
  return cudaGetLastError();
}

cudaError_t launch_loss_total(const float *part, int blocks, double *loss, uint64_t *step, cudaStream_t s) {
  loss_total_kernel<<<1, 32, 0, s>>>(part, blocks, loss, step);
  return cudaGetLastError();
}

cudaError_t launch_unpad(const float *Y, int ldy, size_t n, int fout, float *y, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  unpad_kernel<<<unsigned((n * fout + 255) / 256), 256, 0, s>>>(Y, ldy, n, fout, y);
  return cudaGetLastError();
}

}  // namespace pc
