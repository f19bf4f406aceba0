// pc_greeks.cu -- pathwise sensitivities of the Monte Carlo price.
//
// The kernels and their launch; the tangent evaluator is pc_greeks.cuh.
#include <cstdint>

#include "pc_greeks.cuh"
#include "pc_internal.h"

namespace pc {
namespace {

template <int D, bool WRITE>
__global__ void __launch_bounds__(kBlock) greeks_kernel(const __grid_constant__ PriceArgs a) {
  greeks_tiles<D, WRITE>(a, [&](const uint4 *P, const float *pool, float2 *R, const Rng2 &g, bool live0,
                                bool live1, const float (&Bm)[D * D], const float (&S0)[D],
                                const float (&Lm)[D * D], int gl, float sig_g) {
    return eval_greeks<D>(P, pool, R, a, g, live0, live1, Bm, S0, Lm, gl, sig_g);
  });
}

template <typename K>
cudaError_t set_smem_g(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

}  // namespace

cudaError_t launch_greeks(const PriceArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
  const bool w = a.out_paths != nullptr;
#define GLAUNCH(DD, WW)                                                            \
  do {                                                                             \
    auto k = greeks_kernel<DD, WW>;                                                \
    cudaError_t e = set_smem_g(k, smem);                                           \
    if (e != cudaSuccess) return e;                                                \
    k<<<grid, block, smem, s>>>(a);                                                \
    return cudaGetLastError();                                                     \
  } while (0)
  switch (a.m.d) {
    case 1: if (w) GLAUNCH(1, true); else GLAUNCH(1, false);
    case 2: if (w) GLAUNCH(2, true); else GLAUNCH(2, false);
    case 3: if (w) GLAUNCH(3, true); else GLAUNCH(3, false);
    case 4: if (w) GLAUNCH(4, true); else GLAUNCH(4, false);
    default: return cudaErrorInvalidValue;
  }
#undef GLAUNCH
}

int greeks_blocks_per_sm(int d, int block, size_t smem) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define GOCC(DD)                                                                             \
  set_smem_g(greeks_kernel<DD, false>, smem);                                                \
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, greeks_kernel<DD, false>, block, smem)
  switch (d) {
    case 1: GOCC(1); break;
    case 2: GOCC(2); break;
    case 3: GOCC(3); break;
    case 4: GOCC(4); break;
    default: return 0;
  }
#undef GOCC
  return e == cudaSuccess ? nb : 0;
}

}  // namespace pc
