// Test helper (not part of the library): evaluates the mixed path's fast FP32 helpers
// (qed_common.cuh) element by element, beside CUDA's own atan2f, so that a test can
// check them against FP64 references and error bounds.
#include <cstdint>
#include "../paper_2306_11288_gb300/csrc/qed_common.cuh"

// which: 0 atan01(x), 1 f_atan(x), 2 f_atan2(x, y), 3 atan2f(x, y) (CUDA), 4 f_exp(x),
// 5 f_log(x), 6 sin of f_sincos(x), 7 cos of f_sincos(x), 8 f_rcp(x), 9 f_rsqrt(x)
__global__ void k_fast_math(int which, const float* x, const float* y, float* out, uint64_t n) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a = x[i], b = y[i];
  float r = 0.0f, s = 0.0f, c = 0.0f;
  switch (which) {
    case 0: r = qedk::atan01(a); break;
    case 1: r = qedk::f_atan(a); break;
    case 2: r = qedk::f_atan2(a, b); break;
    case 3: r = atan2f(a, b); break;
    case 4: r = qedk::f_exp(a); break;
    case 5: r = qedk::f_log(a); break;
    case 6: qedk::f_sincos(a, &s, &c); r = s; break;
    case 7: qedk::f_sincos(a, &s, &c); r = c; break;
    case 8: r = qedk::f_rcp(a); break;
    case 9: r = qedk::f_rsqrt(a); break;
    default: r = 0.0f;
  }
  out[i] = r;
}

// x, y, out: device arrays of n floats (y is read only by the two-argument forms, but
// must hold n floats).  Returns a cudaError_t value; 1 for an unknown `which`.
extern "C" int fast_math_eval(int which, const float* x, const float* y, float* out, uint64_t n) {
  if (which < 0 || which > 9) return 1;
  if (n == 0) return 0;
  k_fast_math<<<(unsigned int)((n + 255) / 256), 256>>>(which, x, y, out, n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  return (int)cudaDeviceSynchronize();
}
