// Test helper (not part of the library): Philox4x32-10 blocks from cuRAND's device
// function, the library reference the step's own generator is checked against.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_curand_philox(const uint32_t* ctr, uint64_t key, uint32_t* out, uint64_t n) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint2 k = make_uint2((uint32_t)key, (uint32_t)(key >> 32));
  const uint4 o = curand_Philox4x32_10(c, k);
  out[4 * i] = o.x; out[4 * i + 1] = o.y; out[4 * i + 2] = o.z; out[4 * i + 3] = o.w;
}

// ctr: device n x 4 words; out: device n x 4 words.  Returns a cudaError_t value.
extern "C" int curand_philox_ref(const uint32_t* ctr, uint64_t key, uint32_t* out, uint64_t n) {
  if (n == 0) return 0;
  k_curand_philox<<<(unsigned int)((n + 255) / 256), 256>>>(ctr, key, out, n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  return (int)cudaDeviceSynchronize();
}
