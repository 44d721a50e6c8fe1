// qed_medium.cu -- matter for bremsstrahlung and Bethe-Heitler pair creation (paper Sec.
// III E): the cumulative cross-section tables of a medium, built on the device in FP64, and
// qed_set_medium / the table copy.  The processes themselves run inside the step kernels
// (qed_kernels.cuh: the decisions in the streaming passes, the energies in the event
// kernels).
//
// Cross-sections of Tsai (Rev. Mod. Phys. 46, 815 (1974)), with his screening functions
// phi1,2(gamma), psi1,2(eps) for Thomas-Fermi atoms (Z >= 5) and the Coulomb correction
// f(Z):
//   brems  dsigma/dy = alpha r0^2 D_b / y,  D_b = (4/3 - 4/3 y + y^2) A + (2/3)(1 - y) B,
//   pairs  dsigma/dx = alpha r0^2 D_p,      D_p = (1 - 4/3 x(1-x)) A - (2/3) x(1-x) B,
//   A = Z^2 (phi1 - 4/3 ln Z - 4 f) + Z (psi1 - 8/3 ln Z),  B = Z^2 (phi1 - phi2) + Z (psi1 - psi2),
// gamma = 100 m k / (E E' Z^1/3), eps = 100 m k / (E E' Z^2/3); D < 0 (outside the fits'
// range) counts as 0.  Table layout (the specification both implementations follow): per
// process kNmg rows at ln E uniform on [ln 2, ln 2e6], each the cumulative integral at kNms
// nodes of s in [0, 1], s uniform in the logit ln(v/(1-v)) of the energy fraction between
// its end points (brems y in [k_min/E, 1 - 1/E], pairs x in [1/k, 1 - 1/k]), each node
// interval by 8-point Gauss-Legendre.
#include <cmath>
#include <cstring>

#include "qed_common.cuh"
#include "qed_internal.h"

namespace qedk {

// Gauss-Legendre, 8 points on [-1, 1] (nodes and weights to 16 digits)
__constant__ double c_gl8x[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                                 0.1834346424956498,  0.5255324099163290,  0.7966664774136267,  0.9602898564975363};
__constant__ double c_gl8w[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                                 0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

__device__ double med_brace(int Z, double d, int which, double v) {
  // A, B at screening argument d = m k / (E E')
  const double z13 = cbrt((double)Z), lz = log((double)Z);
  const double g = 100.0 * d / z13, e = 100.0 * d / (z13 * z13);
  const double p1 = 20.863 - 2.0 * log(1.0 + (0.55846 * g) * (0.55846 * g)) -
                    4.0 * (1.0 - 0.6 * exp(-0.9 * g) - 0.4 * exp(-1.5 * g));
  const double p2 = p1 - (2.0 / 3.0) / (1.0 + 6.5 * g + 6.0 * g * g);
  const double q1 = 28.340 - 2.0 * log(1.0 + (3.621 * e) * (3.621 * e)) -
                    4.0 * (1.0 - 0.7 * exp(-8.0 * e) - 0.3 * exp(-29.2 * e));
  const double q2 = q1 - (2.0 / 3.0) / (1.0 + 40.0 * e + 400.0 * e * e);
  const double a2 = (kAlpha * Z) * (kAlpha * Z);
  const double f = a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
  const double zz = (double)Z * Z;
  const double A = zz * (p1 - 4.0 / 3.0 * lz - 4.0 * f) + Z * (q1 - 8.0 / 3.0 * lz);
  const double B = zz * (p1 - p2) + Z * (q1 - q2);
  double D;
  if (which == 0) {   // brems, v = y
    D = (4.0 / 3.0 - 4.0 / 3.0 * v + v * v) * A + (2.0 / 3.0) * (1.0 - v) * B;
  } else {            // pairs, v = x
    const double xx = v * (1.0 - v);
    D = (1.0 - 4.0 / 3.0 * xx) * A - (2.0 / 3.0) * xx * B;
  }
  return D > 0.0 ? D : 0.0;
}

// one block per row (energy node), one thread per node interval; then the block's
// inclusive scan of the interval integrals
__global__ void __launch_bounds__(kNms) k_med_table(int Z, double kmin, int which, double* C) {
  __shared__ double s_w[kNms / 32];
  const int i = blockIdx.x, j = threadIdx.x;   // interval j-1 .. j (thread 0: the row's start)
  const double E = exp(kMgLo + i * ((kMgHi - kMgLo) / (kNmg - 1)));
  const double hs = 1.0 / (kNms - 1);
  const double vlo = which == 0 ? kmin / E : 1.0 / E, vhi = 1.0 - 1.0 / E;
  const bool open = which == 0 ? (vlo < vhi) : (E > 2.0);
  double acc = 0.0;
  if (j > 0 && open) {
    const double tlo = log(vlo / (1.0 - vlo)), thi = log(vhi / (1.0 - vhi));
    for (int q = 0; q < 8; ++q) {
      const double s = (j - 1) * hs + 0.5 * hs * (c_gl8x[q] + 1.0);
      const double t = tlo + s * (thi - tlo);
      const double v = 1.0 / (1.0 + exp(-t)), w = 1.0 / (1.0 + exp(t));
      const double jac = (thi - tlo) * (which == 0 ? w : v * w);
      const double d = which == 0 ? v / (E * (1.0 - v)) : 1.0 / (E * v * (1.0 - v));
      acc += c_gl8w[q] * med_brace(Z, d, which, v) * jac;
    }
    acc *= 0.5 * hs;
  }
  // inclusive scan over the block (warp shuffles, then the warp totals)
  const int lane = j & 31, warp = j >> 5;
  double c = acc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, c, o);
    if (lane >= o) c += t;
  }
  if (lane == 31) s_w[warp] = c;
  __syncthreads();
  if (warp == 0) {
    double w = lane < kNms / 32 ? s_w[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < kNms / 32) s_w[lane] = w;
  }
  __syncthreads();
  C[(size_t)i * kNms + j] = c + (warp ? s_w[warp - 1] : 0.0);
}

// float copies of the row totals (the mixed path's decisions)
__global__ void k_med_totals(const double* C, float* tot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 * kNmg) tot[i] = (float)C[(size_t)i * kNms + kNms - 1];
}

}  // namespace qedk

using namespace qedk;

extern "C" qed_status qed_set_medium(qed_ctx* c, const qed_medium* m, void* stream) {
  const NvtxRange nvtx_range("qed_set_medium");
  if (!c || !c->alive) {
    set_error("qed_set_medium: invalid context");
    return QED_ERR_NOT_INITIALIZED;
  }
  if (!m) {
    c->has_medium = 0;
    return QED_OK;
  }
  if (m->Z < 5 || m->Z > 100 || !(m->n > 0.0) || !std::isfinite(m->n) || !(m->k_min > 0.0) ||
      !std::isfinite(m->k_min) || m->axis < 0 || m->axis > 2 || !(m->lo < m->hi)) {
    set_error("qed_set_medium: need 5 <= Z <= 100 (Tsai's screening functions), n > 0, k_min > 0, "
              "axis 0..2 and lo < hi");
    return QED_ERR_INVALID_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!c->med_buf) {
    cudaError_t e = cudaMalloc(&c->med_buf, kMedBytes);
    if (e != cudaSuccess) {
      set_error("qed_set_medium: cudaMalloc: %s", cudaGetErrorString(e));
      return QED_ERR_CUDA;
    }
  }
  double* C = static_cast<double*>(c->med_buf);
  k_med_table<<<kNmg, kNms, 0, s>>>(m->Z, m->k_min, 0, C);
  k_med_table<<<kNmg, kNms, 0, s>>>(m->Z, m->k_min, 1, C + (size_t)kNmg * kNms);
  k_med_totals<<<(2 * kNmg + 255) / 256, 256, 0, s>>>(C, reinterpret_cast<float*>(C + 2 * (size_t)kNmg * kNms));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error("qed_set_medium: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  c->med = *m;
  c->has_medium = 1;
  return QED_OK;
}

extern "C" qed_status qed_copy_medium_table(qed_ctx* c, double* host, uint64_t cap, uint64_t* len, void* stream) {
  if (!c || !c->alive) {
    set_error("qed_copy_medium_table: invalid context");
    return QED_ERR_NOT_INITIALIZED;
  }
  if (!len) {
    set_error("qed_copy_medium_table: len is NULL");
    return QED_ERR_INVALID_ARG;
  }
  *len = 2ull * kNmg * kNms;
  if (!host) return QED_OK;
  if (!c->has_medium || cap < *len) {
    set_error("qed_copy_medium_table: no medium set, or cap below %llu", (unsigned long long)*len);
    return QED_ERR_INVALID_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(host, c->med_buf, sizeof(double) * *len, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error("qed_copy_medium_table: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  return QED_OK;
}
