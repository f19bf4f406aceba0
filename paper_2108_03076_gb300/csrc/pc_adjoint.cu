// pc_adjoint.cu -- the adjoint sensitivity kernel (pc_adjoint.cuh) and its
// launch.
#include <cstdint>

#include "pc_adjoint.cuh"
#include "pc_internal.h"

namespace pc {
namespace {

template <int D, bool WRITE>
__global__ void __launch_bounds__(kBlock) adjoint_kernel(const __grid_constant__ PriceArgs a, const TapeArgs t) {
  adjoint_tiles<D, WRITE>(a, t, [&](const uint4 *P, const float *pool, float2 *R, const Rng2 &g, bool live0,
                                   bool live1, const float (&Bm)[D * D], const float (&S0)[D],
                                   const float (&Lm)[D * D], Tape &T, int &res) {
    return eval_adjoint<D>(P, pool, R, a, g, live0, live1, Bm, S0, Lm, T, res);
  });
}

template <typename K>
cudaError_t set_smem_a(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

}  // namespace

cudaError_t launch_adjoint(const PriceArgs &a, const TapeArgs &t, int grid, int block, size_t smem,
                           cudaStream_t s) {
  const bool w = a.out_paths != nullptr;
#define ALAUNCH(DD, WW)                                                            \
  do {                                                                             \
    auto k = adjoint_kernel<DD, WW>;                                               \
    cudaError_t e = set_smem_a(k, smem);                                           \
    if (e != cudaSuccess) return e;                                                \
    k<<<grid, block, smem, s>>>(a, t);                                             \
    return cudaGetLastError();                                                     \
  } while (0)
  switch (a.m.d) {
    case 1: if (w) ALAUNCH(1, true); else ALAUNCH(1, false);
    case 2: if (w) ALAUNCH(2, true); else ALAUNCH(2, false);
    case 3: if (w) ALAUNCH(3, true); else ALAUNCH(3, false);
    case 4: if (w) ALAUNCH(4, true); else ALAUNCH(4, false);
    default: return cudaErrorInvalidValue;
  }
#undef ALAUNCH
}

namespace {
int adjoint_occupancy(uint64_t v, int block, size_t smem) {
  const int d = int(v & 0xff);
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define AOCC(DD)                                                                                 \
  do {                                                                                           \
    e = set_smem_a(adjoint_kernel<DD, false>, smem);                                             \
    if (e == cudaSuccess)                                                                        \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, adjoint_kernel<DD, false>, block, smem); \
  } while (0)
  switch (d) {
    case 1: AOCC(1); break;
    case 2: AOCC(2); break;
    case 3: AOCC(3); break;
    case 4: AOCC(4); break;
    default: return 0;
  }
#undef AOCC
  return e == cudaSuccess ? nb : 0;
}
}  // namespace

int adjoint_blocks_per_sm(int d, int block, size_t smem) {
  return occupancy_memo((uint64_t(3) << 32) | uint64_t(d), block, smem, adjoint_occupancy);
}

}  // namespace pc
