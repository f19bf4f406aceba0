// pc_cv.cu -- the delta-hedge control-variate pricing kernel (cv_tiles of
// pc_cv.cuh with the interpreter), and the kernels that turn the network
// into its hedge-ratio tables.
#include <cstdint>

#include "pc_device.cuh"
#include "pc_internal.h"
#include "pc_eval.cuh"
#include "pc_cv.h"
#include "pc_cv.cuh"

namespace pc {
namespace {


template <int D, int MODE>
__global__ void __launch_bounds__(kBlock) cv_kernel(const __grid_constant__ PriceArgs a,
                                                    const __grid_constant__ CvArgs c) {
  using Hook = CvOnline<D, (MODE & kCvGamma) != 0>;
  cv_tiles<D, MODE>(a, c, [&](const uint4 *P, const float *pool, float2 *R, const Rng2 &g, bool live0,
                              bool live1, const float (&Bm)[D * D], const float (&S0)[D], Hook *hook) {
    return eval_path<D, false, Hook>(P, pool, R, a, g, live0, live1, Bm, S0, nullptr, hook);
  });
}

// Network inputs of every table node (cv_feature_row).
__global__ void cv_features_kernel(const CvArgs c, CvFeatureArgs fa, float *X, size_t rows) {
  const size_t r = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (r >= rows) return;
  float f[kCvFeatures];
  cv_feature_row(c, fa, r, rows, f);
  for (int i = 0; i < kCvFeatures; ++i) X[r * kCvFeatures + i] = f[i];
}

// Table entries from the network outputs (value, then one hedge ratio per
// underlying) of the rows above, the ratios of node r at record r (slots
// 0 .. d - 1); the last row's ratios are delta0.
__global__ void cv_scatter_kernel(const float *Y, int out_w, size_t rows, int d, float *tables,
                                  float *delta0) {
  const size_t r = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (r >= rows) return;
  for (int i = 0; i < d; ++i) {
    const float v = Y[r * out_w + 1 + i];
    if (r + 1 < rows) tables[r * kCvRecord + i] = v;
    else delta0[i] = v;
  }
}

// The slopes of every node record from its neighbours' ratios along each
// grid axis: central differences (Delta(a + e_j) - Delta(a - e_j)) / 2, one-
// sided (a difference of 1) on the grid's faces; slots beyond d zeroed.
// Reads slots 0 .. d - 1 and writes the others, in place.
__global__ void cv_slopes_kernel(float *tables, size_t records, int nodes, int G, int d) {
  const size_t r = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (r >= records) return;
  const size_t base = r - r % size_t(nodes);
  const int node = int(r % size_t(nodes));
  float *rec = tables + r * kCvRecord;
  for (int i = d; i < 3; ++i) rec[i] = 0.f;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      float v = 0.f;
      if (i < d && j < d) {
        int stride = 1;
        for (int ax = d - 1; ax > j; --ax) stride *= G;
        const int a = (node / stride) % G;
        const int fwd = a < G - 1 ? node + stride : node, bwd = a > 0 ? node - stride : node;
        const float df = tables[(base + size_t(fwd)) * kCvRecord + i] - tables[(base + size_t(bwd)) * kCvRecord + i];
        v = (a == 0 || a == G - 1) ? df : 0.5f * df;
      }
      rec[3 + 3 * i + j] = v;
    }
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

template <int D>
cudaError_t launch_cv_d(int mode, const PriceArgs &a, const CvArgs &c, int grid, int block, size_t smem,
                        cudaStream_t s) {
#define CVL(MM)                                      \
  do {                                               \
    auto k = cv_kernel<D, MM>;                       \
    cudaError_t e = set_smem(k, smem);               \
    if (e != cudaSuccess) return e;                  \
    k<<<grid, block, smem, s>>>(a, c);               \
    return cudaGetLastError();                       \
  } while (0)
  switch (mode) {
    case 0: CVL(0);
    case kCvGamma: CVL(kCvGamma);
    case kCvPilot: CVL(kCvPilot);
    case kCvPilot | kCvGamma: CVL(kCvPilot | kCvGamma);
    case kCvWrite | kCvGamma: CVL(kCvWrite | kCvGamma);
    default: return cudaErrorInvalidValue;
  }
#undef CVL
}

}  // namespace

int cv_mode(bool write, const CvArgs &c) {
  if (write) return kCvWrite | kCvGamma;
  return (c.use_gamma ? kCvGamma : 0) | (c.pilot ? kCvPilot : 0);
}

cudaError_t launch_cv(const PriceArgs &a, const CvArgs &c, int grid, int block, size_t smem, cudaStream_t s) {
  const int mode = cv_mode(a.out_paths != nullptr, c);
  switch (a.m.d) {
    case 1: return launch_cv_d<1>(mode, a, c, grid, block, smem, s);
    case 2: return launch_cv_d<2>(mode, a, c, grid, block, smem, s);
    case 3: return launch_cv_d<3>(mode, a, c, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

namespace {
int cv_occupancy(uint64_t v, int block, size_t smem) {
  const int d = int(v & 0xff), mode = int((v >> 8) & 0xff);
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define OCC(DD, MM)                                                                      \
  do {                                                                                   \
    e = set_smem(cv_kernel<DD, MM>, smem);                                               \
    if (e == cudaSuccess)                                                                \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cv_kernel<DD, MM>, block, smem); \
  } while (0)
#define OCC_D(DD)                                                      \
  do {                                                                 \
    switch (mode) {                                                    \
      case 0: OCC(DD, 0); break;                                       \
      case kCvGamma: OCC(DD, kCvGamma); break;                         \
      case kCvPilot: OCC(DD, kCvPilot); break;                         \
      default: OCC(DD, kCvPilot | kCvGamma); break;                    \
    }                                                                  \
  } while (0)
  switch (d) {
    case 1: OCC_D(1); break;
    case 2: OCC_D(2); break;
    case 3: OCC_D(3); break;
    default: return 0;
  }
#undef OCC_D
#undef OCC
  return e == cudaSuccess ? nb : 0;
}
}  // namespace

int cv_blocks_per_sm(int d, int block, size_t smem, const CvArgs &c) {
  const int mode = cv_mode(false, c);
  return occupancy_memo((uint64_t(2) << 32) | (uint64_t(mode) << 8) | uint64_t(d), block, smem, cv_occupancy);
}

cudaError_t launch_cv_features(const CvArgs &c, const CvFeatureArgs &fa, float *X, size_t rows,
                               cudaStream_t s) {
  cv_features_kernel<<<unsigned((rows + 127) / 128), 128, 0, s>>>(c, fa, X, rows);
  return cudaGetLastError();
}

cudaError_t launch_cv_scatter(const float *Y, int out_w, size_t rows, int d, float *tables, float *delta0,
                              cudaStream_t s) {
  cv_scatter_kernel<<<unsigned((rows + 127) / 128), 128, 0, s>>>(Y, out_w, rows, d, tables, delta0);
  return cudaGetLastError();
}

cudaError_t launch_cv_slopes(float *tables, size_t records, int nodes, int G, int d, cudaStream_t s) {
  if (records == 0) return cudaSuccess;
  cv_slopes_kernel<<<unsigned((records + 127) / 128), 128, 0, s>>>(tables, records, nodes, G, d);
  return cudaGetLastError();
}

}  // namespace pc
