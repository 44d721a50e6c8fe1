// qed_mlp.cuh -- the learned photon-energy sampler of the NCS events: a 3 -> 64 -> 64 -> 1
// GELU network that maps (ln chi_e, s = S.zeta, one uniform r) to ln u, u = omega/(gamma -
// omega), replacing the two-component inverse-CDF table lookup (the table sampler's
// spin mixture of Eq. Wspin2, inverted as one monotone map of r).
//
// Inference on the tensor cores: a CTA of 128 threads evaluates 128 rows.  Layer 1 (K = 3)
// and the output layer run in FP32 on the CUDA cores; the 64 x 64 hidden layer (94 % of
// the FLOPs) is one tcgen05.mma chain: A = the BF16 hidden activations of the 128 rows and
// B = the BF16 weights, both in shared memory in the canonical no-swizzle K-major layout,
// the FP32 accumulator in tensor memory (64 columns), issued by one thread, completion on
// an mbarrier, read back with tcgen05.ld.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace qedk {

constexpr int kMlpH = 64;                       // hidden width
constexpr int kMlpParams = kMlpH * 3 + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;   // 4481
constexpr int kMlpRows = 128;                   // rows per CTA (= threads = TMEM lanes)

// FP32 parameters (the training master copy and the inference copy of layers 1 and 3) and
// the packed BF16 hidden-layer weights
struct MlpParams {
  float w1[kMlpH][3], b1[kMlpH];
  float w2[kMlpH][kMlpH], b2[kMlpH];
  float w3[kMlpH], b3;
  float pad[3];
  unsigned short w2p[kMlpH * kMlpH];           // BF16, canonical core-matrix layout (see a_offset)
};

// input features and output transform (shared by training and inference)
constexpr float kMlpLnChiLo = -6.907755279f;   // ln 1e-3
constexpr float kMlpLnChiHi = 2.302585093f;    // ln 10
constexpr float kMlpChiLo = 1e-3f, kMlpChiHi = 10.0f;   // trained range of chi_e
__device__ __forceinline__ void mlp_features(float lnchi, float s, float t, float x[3]) {
  x[0] = (2.0f * lnchi - (kMlpLnChiLo + kMlpLnChiHi)) / (kMlpLnChiHi - kMlpLnChiLo);
  x[1] = s;
  x[2] = t * 0.125f;
}
// ln u = ln chi - 3 softplus(-t) + 8 y: the small-u asymptote in t (ln u ~ 3 t) and the
// chi scale, with the network output y as the correction
__device__ __forceinline__ float mlp_base(float lnchi, float t) {
  const float sp = t < -20.0f ? -t : log1pf(expf(-t));
  return lnchi - 3.0f * sp;
}

__device__ __forceinline__ float gelu_f(float x) {
  const float c = 0.7978845608028654f;   // sqrt(2/pi)
  return 0.5f * x * (1.0f + tanhf(c * (x + 0.044715f * x * x * x)));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float c = 0.7978845608028654f;
  const float u = c * (x + 0.044715f * x * x * x);
  const float th = tanhf(u);
  return 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * c * (1.0f + 3.0f * 0.044715f * x * x);
}

// float -> BF16, round to nearest even (finite inputs)
__device__ __forceinline__ unsigned short bf16_rn(float f) {
  const unsigned int b = __float_as_uint(f);
  return (unsigned short)((b + 0x7FFFu + ((b >> 16) & 1u)) >> 16);
}
__device__ __forceinline__ float bf16_to_f(unsigned short h) { return __uint_as_float((unsigned int)h << 16); }

// byte offset of element (row, k) of a [rows x 64] BF16 operand in the canonical
// no-swizzle K-major layout: 8 x 8 core matrices of 128 contiguous bytes (8 rows of 16 B),
// K-adjacent core matrices 128 B apart (LBO), row-adjacent ones 1024 B apart (SBO)
__host__ __device__ __forceinline__ unsigned int a_offset(unsigned int row, unsigned int k) {
  return (row >> 3) * 1024u + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

struct MlpSmem {
  alignas(1024) unsigned char a[kMlpRows * kMlpH * 2];   // hidden activations, BF16 (16 KB)
  alignas(1024) unsigned char w2[kMlpH * kMlpH * 2];     // hidden weights, BF16 (8 KB)
  float w1[kMlpH][3], b1[kMlpH], b2[kMlpH], w3[kMlpH];
  float b3;
  unsigned int taddr;
  alignas(8) unsigned long long bar;
};

__device__ __forceinline__ unsigned int smem_addr(const void* p) { return (unsigned int)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4
// (32-45), the constant 0b001 at bits 46-48, base offset 0, no swizzle
__device__ __forceinline__ unsigned long long smem_desc(unsigned int saddr, unsigned int lbo, unsigned int sbo) {
  unsigned long long d = (unsigned long long)((saddr & 0x3FFFFu) >> 4);
  d |= (unsigned long long)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (unsigned long long)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= 1ull << 46;
  return d;
}
// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 =
// 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr unsigned int kMlpIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kMlpH >> 3) << 17) |
                                   ((unsigned)(kMlpRows >> 4) << 24);

__device__ __forceinline__ void mlp_mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mlp_mbar_try(unsigned long long* bar, unsigned int parity) {
  unsigned int ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: gives up after 2^31 SM clocks (about a second)
static __device__ __noinline__ bool mlp_mbar_wait(unsigned long long* bar, unsigned int parity) {
  const long long t0 = clock64();
  for (unsigned int it = 0; it < (1u << 26); ++it) {
    if (mlp_mbar_try(bar, parity)) return true;
    if (clock64() - t0 > (1ll << 31)) break;
  }
  return false;
}

// All 128 threads: copy the weights, initialise the mbarrier, allocate 64 TMEM columns
// (warp 0).  Must be paired with mlp_teardown on every path.
__device__ __forceinline__ void mlp_setup(MlpSmem& sm, const MlpParams* P) {
  const unsigned int tid = threadIdx.x;
  const uint4* src = reinterpret_cast<const uint4*>(P->w2p);
  uint4* dst = reinterpret_cast<uint4*>(sm.w2);
  for (unsigned int i = tid; i < kMlpH * kMlpH * 2 / 16; i += blockDim.x) dst[i] = src[i];
  for (unsigned int i = tid; i < kMlpH; i += blockDim.x) {
    sm.w1[i][0] = P->w1[i][0]; sm.w1[i][1] = P->w1[i][1]; sm.w1[i][2] = P->w1[i][2];
    sm.b1[i] = P->b1[i]; sm.b2[i] = P->b2[i]; sm.w3[i] = P->w3[i];
  }
  if (tid == 0) {
    sm.b3 = P->b3;
    mlp_mbar_init(&sm.bar);
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.taddr)),
                 "r"((unsigned int)kMlpH)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mlp_teardown(MlpSmem& sm) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.taddr), "r"((unsigned int)kMlpH)
                 : "memory");
  }
}

// One row per thread, all 128 threads (block-uniform call).  Returns the network output y
// for the thread's features x; *ok becomes false (for every thread) if the tensor-core
// chain did not complete within the wait limit.
__device__ __forceinline__ float mlp_rows(MlpSmem& sm, const float x[3], unsigned int& phase, bool* ok) {
  const unsigned int tid = threadIdx.x;
  // layer 1 in FP32, GELU, BF16 into row tid of A
#pragma unroll
  for (int j8 = 0; j8 < kMlpH / 8; ++j8) {
    unsigned int w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      unsigned short v[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int j = j8 * 8 + h * 2 + q;
        const float z = fmaf(sm.w1[j][0], x[0], fmaf(sm.w1[j][1], x[1], fmaf(sm.w1[j][2], x[2], sm.b1[j])));
        v[q] = bf16_rn(gelu_f(z));
      }
      w[h] = (unsigned int)v[0] | ((unsigned int)v[1] << 16);
    }
    *reinterpret_cast<uint4*>(sm.a + a_offset(tid, (unsigned)j8 * 8u)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned int a0 = smem_addr(sm.a), b0 = smem_addr(sm.w2);
#pragma unroll
    for (int k = 0; k < kMlpH / 16; ++k) {
      const unsigned long long ad = smem_desc(a0 + 256u * k, 128u, 1024u);
      const unsigned long long bd = smem_desc(b0 + 256u * k, 128u, 1024u);
      const unsigned int acc = k > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(sm.taddr),
          "l"(ad), "l"(bd), "r"(kMlpIdesc), "r"(acc)
          : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(&sm.bar))
                 : "memory");
  }
  bool done = mlp_mbar_wait(&sm.bar, phase);
  if (!done) done = mlp_mbar_wait(&sm.bar, phase);   // second bounded wait for the chain in flight
  phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // hidden layer accumulators of this row: TMEM lane tid (warp w reads lanes 32w..32w+31)
  float acc[kMlpH];
  const unsigned int lane_base = (tid & ~31u) << 16;
#pragma unroll
  for (int c = 0; c < kMlpH; c += 16) {
    unsigned int r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(sm.taddr + lane_base + (unsigned int)c));
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[c + q] = __uint_as_float(r[q]);
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  float y = sm.b3;
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) y = fmaf(sm.w3[j], gelu_f(acc[j] + sm.b2[j]), y);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  *ok = __syncthreads_and(done) != 0;   // A and TMEM are free for the next rows
  return y;
}

}  // namespace qedk
