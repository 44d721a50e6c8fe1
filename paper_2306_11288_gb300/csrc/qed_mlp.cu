// qed_mlp.cu -- training and evaluation of the learned NCS photon-energy sampler.
//
// Training data: the table sampler itself.  A sample is (ln chi_e ~ U(ln 1e-3, ln 10),
// s ~ U(-1, 1), r ~ U(0, 1); for 1/16 of the samples the logit of r is drawn uniformly
// over [-38, 38] instead, so that the rarely visited tails are fitted) with the
// target ln u = F^{-1}(r) of the spin mixture of
// Eq. Wspin2: F(y) = [w+ F+(y) + w- F-(y)] / (w+ + w-), w+- = (1 +- s)(A -+ B)/2, where
// F+-(y) is the level at which the component's inverse-CDF table reaches y.  F+- and F^{-1}
// are found by bisection on the tables (FP32).
//
// Training: plain FP32 kernels written here.  k_mlp_grad evaluates tiles of 64 samples
// (forward with the BF16 rounding of the hidden layer that inference applies, backward
// with straight-through rounding) and leaves one partial gradient per block; k_mlp_adam
// adds the partials in block order (deterministic) and applies Adam with a cosine learning
// rate.  k_mlp_pack writes the BF16 hidden-layer weights in the tensor-core layout.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "qed_kernels.cuh"
#include "qed_mlp.cuh"

namespace qedk {

// ---- training targets ------------------------------------------------------------------
__device__ float mix_target(const Tabs<float>& tb, float chi, float s, float t) {
  float A, B;
  tb.ncs_rates(chi, A, B);
  const float wp = 0.5f * (1.0f + s) * (A - B), wm = 0.5f * (1.0f - s) * (A + B);
  const float inv_w = 1.0f / (wp + wm);
  const float r = 1.0f / (1.0f + expf(-t));
  // level of component c at which its inverse CDF equals y
  auto level = [&](int c, float y) -> float {
    float lo = (float)kCTLo, hi = (float)kCTHi;
    if (tb.ncs_inv(c, chi, lo) >= y) return 0.0f;
    if (tb.ncs_inv(c, chi, hi) <= y) return 1.0f;
    for (int it = 0; it < 34; ++it) {
      const float m = 0.5f * (lo + hi);
      if (tb.ncs_inv(c, chi, m) < y) lo = m; else hi = m;
    }
    return 1.0f / (1.0f + expf(-0.5f * (lo + hi)));
  };
  float ylo = fminf(tb.ncs_inv(0, chi, (float)kCTLo), tb.ncs_inv(1, chi, (float)kCTLo));
  float yhi = fmaxf(tb.ncs_inv(0, chi, (float)kCTHi), tb.ncs_inv(1, chi, (float)kCTHi));
  for (int it = 0; it < 40; ++it) {
    const float y = 0.5f * (ylo + yhi);
    const float F = (wp * level(0, y) + wm * level(1, y)) * inv_w;
    if (F < r) ylo = y; else yhi = y;
  }
  return 0.5f * (ylo + yhi);
}

// sample i: features and the regression target (ln u - base) / 8
__global__ void k_mlp_gen(const float* tables, unsigned long long seed, unsigned long long first,
                          unsigned long long n, float4* out) {
  const Tabs<float> tb = tabs_global<float>(tables);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long g = first + i;
    const U4 o = philox10((uint32_t)g, (uint32_t)(g >> 32), 0x4D4C5053u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float lnchi = kMlpLnChiLo + (kMlpLnChiHi - kMlpLnChiLo) * ((float)(o.c >> 8) * 0x1p-24f);
    const float s = 2.0f * ((float)(o.d >> 8) * 0x1p-24f) - 1.0f;
    const double r = ((double)(((uint64_t)(o.a >> 5) << 26) | (uint64_t)(o.b >> 6)) + 0.5) * 0x1p-53;
    double td;
    if ((o.c & 0xFFu) < 16u) {
      td = kCTLo + (kCTHi - kCTLo) * r;   // 1/16 of the rows: the logit uniform over its range (tails)
    } else {
      td = log(r) - log1p(-r);            // the rest: the logit of a uniform level
    }
    td = td < kCTLo ? kCTLo : (td > kCTHi ? kCTHi : td);
    const float t = (float)td;
    float x[3];
    mlp_features(lnchi, s, t, x);
    const float y = mix_target(tb, expf(lnchi), s, t);
    out[i] = make_float4(x[0], x[1], x[2], (y - mlp_base(lnchi, t)) * 0.125f);
  }
}

// table-sampler target for given (ln chi, s, r) (test and error-measurement entry)
__global__ void k_mlp_target(const float* tables, const float* in, float* out, unsigned long long n) {
  const Tabs<float> tb = tabs_global<float>(tables);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float lnchi = in[3 * i], s = in[3 * i + 1];
    const double r = in[3 * i + 2];
    double td = log(r) - log1p(-r);
    td = td < kCTLo ? kCTLo : (td > kCTHi ? kCTHi : td);
    out[i] = mix_target(tb, expf(lnchi), s, (float)td);
  }
}

// ---- training ---------------------------------------------------------------------------
constexpr int kTrainTile = 64;      // samples per tile
constexpr int kTrainThreads = 256;

struct TrainSmem {
  float w1[kMlpH][3], b1[kMlpH], w2q[kMlpH][kMlpH + 1], b2[kMlpH], w3[kMlpH];
  float b3;
  float x[kTrainTile][3], tgt[kTrainTile], dy[kTrainTile];
  float g1[kTrainTile][kMlpH + 1];   // gelu'(z1)
  float h1q[kTrainTile][kMlpH + 1];  // BF16-rounded gelu(z1)
  float g2[kTrainTile][kMlpH + 1];   // gelu'(z2), then dZ2
  float h2[kTrainTile][kMlpH + 1];   // gelu(z2)
};

// partial gradients of block b: grad[b * kMlpParams + p], parameters in MlpParams order
__global__ void __launch_bounds__(kTrainThreads) k_mlp_grad(const MlpParams* P, const float4* data,
                                                           unsigned long long n, float inv_batch, float* grad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int tid = threadIdx.x;
  for (int i = tid; i < kMlpH; i += blockDim.x) {
    S.w1[i][0] = P->w1[i][0]; S.w1[i][1] = P->w1[i][1]; S.w1[i][2] = P->w1[i][2];
    S.b1[i] = P->b1[i]; S.b2[i] = P->b2[i]; S.w3[i] = P->w3[i];
  }
  for (int i = tid; i < kMlpH * kMlpH; i += blockDim.x) {
    const float w = P->w2[i / kMlpH][i % kMlpH];
    S.w2q[i / kMlpH][i % kMlpH] = bf16_to_f(bf16_rn(w));
  }
  if (tid == 0) S.b3 = P->b3;
  __syncthreads();
  // gradient accumulators owned by this thread: W2 entries tid + 256 k (16 of them), and
  // one of {W1 (192), b1, b2, w3} entries (tid < 192 + 64 * 3 is split over two passes)
  float gw2[kMlpH * kMlpH / kTrainThreads];
#pragma unroll
  for (int k = 0; k < kMlpH * kMlpH / kTrainThreads; ++k) gw2[k] = 0.0f;
  float gA = 0.0f, gB = 0.0f, gb3 = 0.0f;   // gA: W1 entry tid (tid < 192) ; gB: b1/b2/w3 entry
  const unsigned long long ntiles = (n + kTrainTile - 1) / kTrainTile;
  for (unsigned long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const unsigned long long base = tile * kTrainTile;
    for (int m = tid; m < kTrainTile; m += blockDim.x) {
      const bool ok = base + m < n;
      const float4 d = ok ? data[base + m] : make_float4(0.f, 0.f, 0.f, 0.f);
      S.x[m][0] = d.x; S.x[m][1] = d.y; S.x[m][2] = d.z; S.tgt[m] = d.w;
      S.dy[m] = ok ? 1.0f : 0.0f;   // mask, replaced by dL/dy below
    }
    __syncthreads();
    // layer 1
    for (int e = tid; e < kTrainTile * kMlpH; e += blockDim.x) {
      const int m = e / kMlpH, j = e % kMlpH;
      const float z = fmaf(S.w1[j][0], S.x[m][0], fmaf(S.w1[j][1], S.x[m][1], fmaf(S.w1[j][2], S.x[m][2], S.b1[j])));
      S.g1[m][j] = gelu_grad_f(z);
      S.h1q[m][j] = bf16_to_f(bf16_rn(gelu_f(z)));
    }
    __syncthreads();
    // layer 2
    for (int e = tid; e < kTrainTile * kMlpH; e += blockDim.x) {
      const int m = e / kMlpH, j = e % kMlpH;
      float z = S.b2[j];
#pragma unroll 16
      for (int k = 0; k < kMlpH; ++k) z = fmaf(S.h1q[m][k], S.w2q[j][k], z);
      S.g2[m][j] = gelu_grad_f(z);
      S.h2[m][j] = gelu_f(z);
    }
    __syncthreads();
    // output and dL/dy (mean squared error over the batch)
    if (tid < kTrainTile) {
      const int m = tid;
      float y = S.b3;
      for (int j = 0; j < kMlpH; ++j) y = fmaf(S.w3[j], S.h2[m][j], y);
      S.dy[m] = S.dy[m] * 2.0f * (y - S.tgt[m]) * inv_batch;
      gb3 += S.dy[m];
    }
    __syncthreads();
    // w3 gradient, then dZ2 = dy w3 gelu'(z2) in place of g2
    if (tid >= 128 && tid < 128 + kMlpH) {
      const int j = tid - 128;
      float g = 0.0f;
      for (int m = 0; m < kTrainTile; ++m) g = fmaf(S.dy[m], S.h2[m][j], g);
      gB += g;   // thread 128 + j owns w3[j]
    }
    __syncthreads();
    for (int e = tid; e < kTrainTile * kMlpH; e += blockDim.x) {
      const int m = e / kMlpH, j = e % kMlpH;
      S.g2[m][j] *= S.dy[m] * S.w3[j];
    }
    __syncthreads();
    // W2 gradient (straight through the BF16 rounding): dZ2^T h1q; b2 gradient
#pragma unroll
    for (int k = 0; k < kMlpH * kMlpH / kTrainThreads; ++k) {
      const int e = tid + k * kTrainThreads;
      const int j = e / kMlpH, i = e % kMlpH;
      float g = 0.0f;
      for (int m = 0; m < kTrainTile; ++m) g = fmaf(S.g2[m][j], S.h1q[m][i], g);
      gw2[k] += g;
    }
    if (tid >= 64 && tid < 64 + kMlpH) {
      const int j = tid - 64;
      float g = 0.0f;
      for (int m = 0; m < kTrainTile; ++m) g += S.g2[m][j];
      gB += g;   // thread 64 + j owns b2[j]
    }
    // dZ1 = (dZ2 W2q) gelu'(z1), into g1
    __syncthreads();
    for (int e = tid; e < kTrainTile * kMlpH; e += blockDim.x) {
      const int m = e / kMlpH, i = e % kMlpH;
      float g = 0.0f;
#pragma unroll 16
      for (int j = 0; j < kMlpH; ++j) g = fmaf(S.g2[m][j], S.w2q[j][i], g);
      S.h1q[m][i] = g * S.g1[m][i];   // dZ1 (h1q no longer needed)
    }
    __syncthreads();
    // W1 and b1 gradients
    if (tid < kMlpH * 3) {
      const int j = tid / 3, c = tid % 3;
      float g = 0.0f;
      for (int m = 0; m < kTrainTile; ++m) g = fmaf(S.h1q[m][j], S.x[m][c], g);
      gA += g;
    }
    if (tid < kMlpH) {
      float g = 0.0f;
      for (int m = 0; m < kTrainTile; ++m) g += S.h1q[m][tid];
      gB += g;   // thread j owns b1[j]
    }
    __syncthreads();
  }
  // parameter order: w1 (192), b1 (64), w2 (4096), b2 (64), w3 (64), b3
  float* out = grad + (size_t)blockIdx.x * kMlpParams;
  if (tid < kMlpH * 3) out[tid] = gA;
  if (tid < kMlpH) out[192 + tid] = gB;
#pragma unroll
  for (int k = 0; k < kMlpH * kMlpH / kTrainThreads; ++k) out[256 + tid + k * kTrainThreads] = gw2[k];
  if (tid >= 64 && tid < 128) out[256 + 4096 + (tid - 64)] = gB;
  if (tid >= 128 && tid < 192) out[256 + 4096 + 64 + (tid - 128)] = gB;
  // b3: sum over the threads that own output rows
  __shared__ float s_b3[kTrainThreads];
  s_b3[tid] = gb3;
  __syncthreads();
  if (tid == 0) {
    float g = 0.0f;
    for (int k = 0; k < kTrainTile; ++k) g += s_b3[k];
    out[kMlpParams - 1] = g;
  }
}

// Adam over the flat parameter vector (MlpParams order), gradients summed over blocks in order
__global__ void k_mlp_adam(MlpParams* P, float* m, float* v, const float* grad, int nblk, float lr, float b1t,
                           float b2t) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  float g = 0.0f;
  for (int b = 0; b < nblk; ++b) g += grad[(size_t)b * kMlpParams + p];
  float* w = reinterpret_cast<float*>(P);
  const float beta1 = 0.9f, beta2 = 0.999f;
  const float mm = beta1 * m[p] + (1.0f - beta1) * g;
  const float vv = beta2 * v[p] + (1.0f - beta2) * g * g;
  m[p] = mm;
  v[p] = vv;
  w[p] -= lr * (mm / (1.0f - b1t)) / (sqrtf(vv / (1.0f - b2t)) + 1e-8f);
}

__global__ void k_mlp_pack(MlpParams* P) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kMlpH * kMlpH; e += gridDim.x * blockDim.x) {
    const int n = e / kMlpH, k = e % kMlpH;
    P->w2p[a_offset((unsigned)n, (unsigned)k) / 2] = bf16_rn(P->w2[n][k]);
  }
}

// ---- tensor-core evaluation of given inputs ----------------------------------------------
__global__ void __launch_bounds__(kMlpRows) k_mlp_eval(const MlpParams* P, const float* in, float* out,
                                                      unsigned long long n, unsigned int* status) {
  __shared__ MlpSmem sm;
  mlp_setup(sm, P);
  unsigned int phase = 0;
  const unsigned long long nchunk = (n + kMlpRows - 1) / kMlpRows;
  for (unsigned long long c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const unsigned long long i = c * kMlpRows + threadIdx.x;
    const bool valid = i < n;
    const float lnchi = valid ? in[3 * i] : 0.0f, s = valid ? in[3 * i + 1] : 0.0f;
    const double r = valid ? (double)in[3 * i + 2] : 0.5;
    double td = log(r) - log1p(-r);
    td = td < kCTLo ? kCTLo : (td > kCTHi ? kCTHi : td);
    const float t = (float)td;
    float x[3];
    mlp_features(lnchi, s, t, x);
    bool ok;
    const float y = mlp_rows(sm, x, phase, &ok);
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(status, QED_STATUS_TIMEOUT);
      break;
    }
    if (valid) out[i] = mlp_base(lnchi, t) + 8.0f * y;
  }
  mlp_teardown(sm);
}

}  // namespace qedk

using namespace qedk;

#define MFAIL(code, ...)     \
  do {                       \
    set_error(__VA_ARGS__);  \
    return code;             \
  } while (0)
#define MCK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) MFAIL(QED_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static qed_ctx* owner_of(qed_ctx* c) { return c->owner ? c->owner : c; }

static qed_status mlp_alloc(qed_ctx* c) {
  if (c->mlp) return QED_OK;
  MCK(cudaMalloc(&c->mlp, sizeof(MlpParams)));
  MCK(cudaMemset(c->mlp, 0, sizeof(MlpParams)));
  return QED_OK;
}

extern "C" qed_status qed_mlp_set_params(qed_ctx* ctx, const float* host, void* stream) {
  if (!ctx || !ctx->alive) MFAIL(QED_ERR_NOT_INITIALIZED, "qed_mlp_set_params: invalid context");
  if (!host) MFAIL(QED_ERR_INVALID_ARG, "qed_mlp_set_params: host is NULL");
  qed_ctx* o = owner_of(ctx);
  const qed_status r = mlp_alloc(o);
  if (r != QED_OK) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MCK(cudaMemcpyAsync(o->mlp, host, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s));
  k_mlp_pack<<<16, 256, 0, s>>>(static_cast<MlpParams*>(o->mlp));
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(s));
  o->mlp_ready = 1;
  return QED_OK;
}

extern "C" qed_status qed_mlp_get_params(qed_ctx* ctx, float* host, void* stream) {
  if (!ctx || !ctx->alive) MFAIL(QED_ERR_NOT_INITIALIZED, "qed_mlp_get_params: invalid context");
  qed_ctx* o = owner_of(ctx);
  if (!host || !o->mlp_ready) MFAIL(QED_ERR_INVALID_ARG, "qed_mlp_get_params: no parameters (train or set first)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MCK(cudaMemcpyAsync(host, o->mlp, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  return QED_OK;
}

extern "C" qed_status qed_mlp_train(qed_ctx* ctx, uint64_t n_samples, uint32_t batch, uint64_t seed, void* stream) {
  if (!ctx || !ctx->alive) MFAIL(QED_ERR_NOT_INITIALIZED, "qed_mlp_train: invalid context");
  if (n_samples < batch || batch < kTrainTile || batch > (1u << 22))
    MFAIL(QED_ERR_INVALID_ARG, "qed_mlp_train: need 64 <= batch <= 2^22 and batch <= n_samples");
  qed_ctx* o = owner_of(ctx);
  qed_status r = mlp_alloc(o);
  if (r != QED_OK) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int sms = 0;
  MCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o->device));
  // initial parameters: uniform(+-sqrt(6 / (fan_in + fan_out))), zero biases
  std::vector<float> h(kMlpParams, 0.0f);
  std::mt19937_64 gen(seed ^ 0x9E3779B97F4A7C15ull);
  auto fill = [&](int off, int cnt, float lim) {
    std::uniform_real_distribution<float> u(-lim, lim);
    for (int i = 0; i < cnt; ++i) h[off + i] = u(gen);
  };
  fill(0, kMlpH * 3, std::sqrt(6.0f / (3 + kMlpH)));
  fill(256, kMlpH * kMlpH, std::sqrt(6.0f / (2 * kMlpH)));
  fill(256 + 4096 + 64, kMlpH, std::sqrt(6.0f / (kMlpH + 1)));
  MCK(cudaMemcpyAsync(o->mlp, h.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s));
  // buffers: samples, Adam moments, partial gradients
  const int nblk = std::min<int>(sms * 2, (int)((batch + kTrainTile - 1) / kTrainTile));
  float4* data = nullptr;
  float *m = nullptr, *v = nullptr, *grad = nullptr;
  // samples are generated in chunks of whole batches (about 16M samples, 256 MB at a time)
  const unsigned long long per_chunk = std::max<unsigned long long>(1, (1ull << 24) / batch);
  const unsigned long long chunk = per_chunk * batch;
  cudaError_t e = cudaMalloc(&data, sizeof(float4) * chunk);
  if (e == cudaSuccess) e = cudaMalloc(&m, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&v, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&grad, sizeof(float) * kMlpParams * nblk);
  if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, sizeof(float) * kMlpParams, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(float) * kMlpParams, s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
  const unsigned long long steps = n_samples / batch;
  const float lr0 = 3e-3f, lr_min = 2e-5f;
  double b1t = 1.0, b2t = 1.0;
  for (unsigned long long step = 0; step < steps && e == cudaSuccess; ++step) {
    const unsigned long long first = step * batch, off = first % chunk;
    if (off == 0)
      k_mlp_gen<<<sms * 8, 256, 0, s>>>(o->tab32, seed, first, std::min<unsigned long long>(chunk, steps * batch - first),
                                        data);
    k_mlp_grad<<<nblk, kTrainThreads, sizeof(TrainSmem), s>>>(static_cast<MlpParams*>(o->mlp), data + off, batch,
                                                               1.0f / (float)batch, grad);
    b1t *= 0.9;
    b2t *= 0.999;
    const double frac = (double)step / (double)std::max<unsigned long long>(steps - 1, 1);
    const float lr = (float)(lr_min + 0.5 * (lr0 - lr_min) * (1.0 + std::cos(3.141592653589793 * frac)));
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(static_cast<MlpParams*>(o->mlp), m, v, grad, nblk, lr,
                                                        (float)b1t, (float)b2t);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_mlp_pack<<<16, 256, 0, s>>>(static_cast<MlpParams*>(o->mlp));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(data);
  cudaFree(m);
  cudaFree(v);
  cudaFree(grad);
  if (e != cudaSuccess) MFAIL(QED_ERR_CUDA, "qed_mlp_train: %s", cudaGetErrorString(e));
  o->mlp_ready = 1;
  return QED_OK;
}

extern "C" qed_status qed_mlp_eval(qed_ctx* ctx, const float* dev_in, float* dev_out, uint64_t n, void* stream) {
  if (!ctx || !ctx->alive) MFAIL(QED_ERR_NOT_INITIALIZED, "qed_mlp_eval: invalid context");
  qed_ctx* o = owner_of(ctx);
  if (!o->mlp_ready) MFAIL(QED_ERR_NOT_INITIALIZED, "qed_mlp_eval: the sampler has no parameters (train or set)");
  if ((!dev_in || !dev_out) && n) MFAIL(QED_ERR_INVALID_ARG, "qed_mlp_eval: NULL buffers");
  if (!n) return QED_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int sms = 0;
  MCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o->device));
  const unsigned long long want = (n + kMlpRows - 1) / kMlpRows;
  const int grid = (int)std::min<unsigned long long>(want, (unsigned long long)sms * 4);
  k_mlp_eval<<<grid, kMlpRows, 0, s>>>(static_cast<const MlpParams*>(o->mlp), dev_in, dev_out, n,
                                       &o->st->status);
  MCK(cudaGetLastError());
  return QED_OK;
}

extern "C" qed_status qed_mlp_target(qed_ctx* ctx, const float* dev_in, float* dev_out, uint64_t n, void* stream) {
  if (!ctx || !ctx->alive) MFAIL(QED_ERR_NOT_INITIALIZED, "qed_mlp_target: invalid context");
  if ((!dev_in || !dev_out) && n) MFAIL(QED_ERR_INVALID_ARG, "qed_mlp_target: NULL buffers");
  if (!n) return QED_OK;
  qed_ctx* o = owner_of(ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_mlp_target<<<(unsigned)std::min<unsigned long long>((n + 255) / 256, 4096), 256, 0, s>>>(o->tab32, dev_in, dev_out, n);
  MCK(cudaGetLastError());
  return QED_OK;
}
