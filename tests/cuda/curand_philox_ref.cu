// Test helper: cuRAND's device-side Philox4x32-10 (curand_Philox4x32_10 from
// curand_kernel.h) applied to a list of counters, as an independent
// reference for the engine's own Philox implementation and for the oracle.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_philox_kernel(const uint4 *ctr, uint32_t k0, uint32_t k1, uint4 *out,
                                     size_t n) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(ctr[i], make_uint2(k0, k1));
}

extern "C" int curand_philox_ref(const uint32_t *d_ctr, uint32_t k0, uint32_t k1,
                                 uint32_t *d_out, size_t n) {
  if (n == 0) return 0;
  curand_philox_kernel<<<unsigned((n + 255) / 256), 256>>>(
      reinterpret_cast<const uint4 *>(d_ctr), k0, k1, reinterpret_cast<uint4 *>(d_out), n);
  return int(cudaDeviceSynchronize());
}
