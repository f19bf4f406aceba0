// pc_mlp.h -- device-side pieces of the learned control variate's network
// (pc_mlp.cu) and their host launchers.  Private to the library.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace pc {

#ifdef __CUDACC__
// softplus(z) = max(z, 0) + log(1 + u), u = exp(-|z|) in (0, 1]: u from the
// SFU (ex2), log(1 + u) = u p(u) with p a degree-6 polynomial fitted here by
// least squares to log(1 + u) / u on Chebyshev points of [0, 1] (relative
// error of u p(u) below 1.5e-6 in FP32): one SFU operation instead of two,
// far inside the BF16 rounding (2^-9 relative) of the stored activation.
__device__ __forceinline__ float softplus_fast(float z) {
  float u;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(u) : "f"(-1.4426950408889634f * fabsf(z)));
  float p = 0.014202825725078583f;
  p = fmaf(p, u, -0.06658805161714554f);
  p = fmaf(p, u, 0.14943458139896393f);
  p = fmaf(p, u, -0.23514863848686218f);
  p = fmaf(p, u, 0.3311205208301544f);
  p = fmaf(p, u, -0.4998719096183777f);
  p = fmaf(p, u, 0.9999987483024597f);
  return fmaxf(z, 0.f) + u * p;
}
#endif

// GEMM epilogues of mlp_gemm.
constexpr int kEpiBiasSoftplus = 0;  // Cb = bf16(softplus(acc + bias))
constexpr int kEpiBias = 1;          // Cf = acc + bias (FP32)
constexpr int kEpiDSoftplus = 2;     // Cb = bf16(acc * (1 - exp(-aux)))
constexpr int kEpiPartial = 3;       // Cf[z] = acc over this k split (FP32)

// C[M, N] = op(A) op(B) over K; M, N multiples of 64, K and k_split
// multiples of 32; leading dimensions in elements, multiples of 8.
struct GemmArgs {
  const __nv_bfloat16 *A;
  int lda;
  const __nv_bfloat16 *B;
  int ldb;
  int M, N, K;
  int k_split;                  // k range per blockIdx.z
  const float *bias;            // [N] (bias epilogues)
  const __nv_bfloat16 *aux;     // stored activations (kEpiDSoftplus)
  int ldaux;
  __nv_bfloat16 *Cb;            // BF16 output
  float *Cf;                    // FP32 output (partials: [splits][M][ldc])
  int ldc;
};

enum GemmKind { kGemmForward, kGemmDataGrad, kGemmWeightGrad };
cudaError_t launch_gemm(GemmKind kind, int epi, const GemmArgs &g, int splits, cudaStream_t s);

// The products on the tcgen05 tensor cores (pc_mlp_tc.cu), operands staged
// by TMA in the 128-byte swizzled layout: kGemmForward (A [M][K] and B [N][K]
// K-major; epilogues kEpiBiasSoftplus, kEpiBias), kGemmDataGrad (A [M][K]
// K-major, B = W [K][N] N-major; kEpiDSoftplus), kGemmWeightGrad (A = dZ
// [K][M] M-major, B = the layer input [K][N] N-major; kEpiPartial, split over
// K in k_split ranges by blockIdx.z).  K and k_split multiples of 64, M of
// 64, N = 64 or a multiple of 128.  *status |= 4 when a bounded wait
// expires.  gemm_tc_init (once, outside stream capture):
// cudaErrorNotSupported on devices or drivers without them.
// The TMA descriptors of a product's operands (encoded once per buffer and
// shape on the host; kernel parameters by value).
struct TcMaps {
  CUtensorMap a, b;
};
cudaError_t gemm_tc_init();
bool gemm_tc_supported(GemmKind kind, const GemmArgs &g);
bool make_tc_maps(GemmKind kind, const GemmArgs &g, TcMaps &m);
// withhold: failure test (the producer withholds its first copies and the
// bounded waits expire after about 10 ms)
cudaError_t launch_gemm_tc(GemmKind kind, int epi, const GemmArgs &g, const TcMaps &m, int splits,
                           int32_t *status, cudaStream_t s, bool withhold = false);

// The control variate's hedge tables in one launch (cv_tables_tc): per
// 128-row tile, the network inputs of the table rows (cv_feature_row) go to
// shared memory, every layer's product runs on tcgen05 from there (weights
// streamed by TMA, the accumulator in TMEM), the hidden activations return
// to shared memory as the next layer's operand, and the last layer's hedge
// ratios go to the tables (row r < rows - 1: tables[12 r + i]; the last row:
// delta0).  Networks of up to kCvNetMaxLayers layers, input and output
// padded to 64, hidden widths multiples of 64 up to 256.
constexpr int kCvNetMaxLayers = 4;
struct CvTablesTc {
  CUtensorMap w[kCvNetMaxLayers];       // layer l's BF16 weights [wp[l+1]][wp[l]], box 64 x wp[l+1]
  const float *bias[kCvNetMaxLayers];   // [wp[l+1]], zero padded
  int L;
  int wp[kCvNetMaxLayers + 1];
  size_t rows;
  float *tables, *delta0;
  int32_t *status;                      // |= 4 when a bounded wait expires
  // failure test: the producer withholds the first weight chunk's copy, so
  // the waits on it expire (after about 10 ms) and the kernel takes its
  // abort path
  int withhold;
};
bool cv_tables_tc_shape(int L, const int *wp);
bool make_weight_map(CUtensorMap &m, const __nv_bfloat16 *w, int n_out, int n_in);
cudaError_t launch_cv_tables_tc(const CvTablesTc &t, const struct CvArgs &c, const struct CvFeatureArgs &fa,
                                cudaStream_t s);
// x [n, fin] FP32 -> X [rows, ld] BF16, zero beyond n rows / fin columns.
cudaError_t launch_to_bf16(const float *x, size_t n, int fin, __nv_bfloat16 *X, size_t rows, int ld,
                           cudaStream_t s);
// Gather a minibatch: rows idx = Philox(seed, step, b) mod n_data of
// x [n_data, fin] and t [n_data, fout] into X (BF16, padded) and T (FP32).
cudaError_t launch_gather(const float *x, const float *t, size_t n_data, int fin, int fout,
                          const uint64_t *step, uint32_t seed_lo, uint32_t seed_hi, size_t batch,
                          __nv_bfloat16 *X, int ldx, float *T, cudaStream_t s);
// Weighted squared-error loss of Y [rows, ldy] (FP32) against T [n, fout]:
// dY = (2 / n) w (Y - T) as BF16 [rows, ldd] (zero beyond n rows / fout
// columns), per-block loss partials into part[blocks].
cudaError_t launch_loss(const float *Y, int ldy, const float *T, const float *w, size_t n, int fout,
                        size_t rows, __nv_bfloat16 *dY, int ldd, float *part, int blocks,
                        cudaStream_t s);
int loss_blocks(size_t rows);
// out[i] = sum_s part[s * stride + i], s < splits, in order; i < count.
cudaError_t launch_split_sum(const float *part, int splits, size_t stride, size_t count, float *out,
                             cudaStream_t s);
// Column sums of dZ [rows, ld] (BF16) for columns < cols into out (FP32),
// in a fixed order (row chunks, then the chunk partials).
cudaError_t launch_colsum(const __nv_bfloat16 *dZ, size_t rows, int ld, int cols, float *scratch,
                          float *out, cudaStream_t s);
// Adam over flat parameters p (FP32) with gradient g; moments m, v; bf16
// copy pb; bias corrections for step *step + 1.
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, size_t n,
                        uint64_t *step, float lr, float b1, float b2, float eps, cudaStream_t s);
// Sum of part[0..blocks) into *loss (FP64) in order; then ++*step if step.
cudaError_t launch_loss_total(const float *part, int blocks, double *loss, uint64_t *step, cudaStream_t s);
// y [n, fout] FP32 from Y [rows, ldy].
cudaError_t launch_unpad(const float *Y, int ldy, size_t n, int fout, float *y, cudaStream_t s);

}  // namespace pc
