// qed_diag.cu -- end-of-run observables of one particle set: spectra in ln(energy) and
// detector maps in (x, y), each bin holding sum w, sum w o (o = spin vector for leptons,
// Stokes parameters in the detection basis for photons, paper Sec. IV post-processing
// with the basis change of Eq. (rotation)) and the count.
//
// k_diag: every block accumulates its grid-stride share of the set in a shared-memory
// histogram (FP64) and keeps the totals per thread with Neumaier compensation; its
// partial histogram goes to scratch.  k_diag_final: one thread per output value adds the
// blocks' partials in block order with Neumaier compensation.
#include <cmath>
#include <cstring>

#include "qed_common.cuh"
#include "qed_internal.h"

namespace qedk {

constexpr int kDiagThreads = 256;
constexpr int kDiagMaxBins = 1024;
constexpr int kDiagVals = 5;   // sum w, sum w o1, sum w o2, sum w o3, count

struct DiagArgs {
  const double *x, *y, *z;
  const void *px, *py, *pz, *s1, *s2, *s3, *theta, *w;
  const unsigned long long* n_live;
  int photon, kind, nx, ny;
  double lnlo, inv_dln;          // spectrum: bins in ln(energy)
  double lo_x, lo_y, inv_dx, inv_dy;   // detector: bins in x, y
  double ref[3];
  double* partial;               // [grid][len]
  int len;                       // kDiagVals * (nbins + 1) + 2
};

struct Neumaier {
  double s = 0.0, c = 0.0;
  __device__ void add(double v) {
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  __device__ double value() const { return s + c; }
};

template <typename R>
__device__ __forceinline__ double ldd(const void* p, unsigned long long i) {
  return (double)reinterpret_cast<const R*>(p)[i];
}

// Stokes parameters of a photon in the detection basis (d1, d2 = n x d1), rotated from
// the stored basis P1 = cos(theta) e1 + sin(theta) e2 of the canonical frame of n.
__device__ void detector_stokes(const double n[3], double theta, const double xi[3], const double ref[3],
                                double out[3]) {
  // canonical frame: e1 = unit(y x n) (unit(n x x) near +-y), e2 = n x e1
  double a = n[2], b = 0.0, c = -n[0];
  double m2 = a * a + c * c;
  if (m2 < 1e-20) { a = 0.0; b = n[2]; c = -n[1]; m2 = b * b + c * c; }
  const double inv = 1.0 / sqrt(m2);
  const double e1[3] = {a * inv, b * inv, c * inv};
  const double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
  const double rn = ref[0] * n[0] + ref[1] * n[1] + ref[2] * n[2];
  const double d1[3] = {ref[0] - rn * n[0], ref[1] - rn * n[1], ref[2] - rn * n[2]};
  const double dd = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2];
  const double thd = dd < 1e-20 ? 0.0 : atan2(d1[0] * e2[0] + d1[1] * e2[1] + d1[2] * e2[2],
                                              d1[0] * e1[0] + d1[1] * e1[1] + d1[2] * e1[2]);
  double s2, c2;
  sincos(2.0 * (thd - theta), &s2, &c2);
  out[0] = xi[0] * c2 - xi[2] * s2;
  out[1] = xi[1];
  out[2] = xi[0] * s2 + xi[2] * c2;
}

template <typename R>
__global__ void __launch_bounds__(kDiagThreads) k_diag(DiagArgs a) {
  __shared__ double s_h[kDiagVals * (kDiagMaxBins + 1) + 2];
  __shared__ double s_red[kDiagThreads];
  const int nb = a.nx * a.ny;
  for (int k = threadIdx.x; k < a.len; k += blockDim.x) s_h[k] = 0.0;
  __syncthreads();
  Neumaier tot[kDiagVals + 2];
  const unsigned long long n = *a.n_live;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const double w = ldd<R>(a.w, i);
    const double p[3] = {ldd<R>(a.px, i), ldd<R>(a.py, i), ldd<R>(a.pz, i)};
    const double s[3] = {ldd<R>(a.s1, i), ldd<R>(a.s2, i), ldd<R>(a.s3, i)};
    const double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    double o[3] = {s[0], s[1], s[2]};
    double energy;
    if (a.photon) {
      energy = sqrt(p2);
      if (energy > 0.0) {
        const double nn[3] = {p[0] / energy, p[1] / energy, p[2] / energy};
        detector_stokes(nn, ldd<R>(a.theta, i), s, a.ref, o);
      }
    } else {
      energy = sqrt(1.0 + p2);
    }
    int bin = -1;        // -1 below, -2 above / outside
    if (a.kind == QED_DIAG_SPECTRUM) {
      const double t = energy > 0.0 ? (log(energy) - a.lnlo) * a.inv_dln : -1.0;
      if (t < 0.0) bin = -1;
      else if (t >= (double)a.nx) bin = -2;
      else bin = min((int)t, a.nx - 1);
    } else {
      const double tx = (a.x[i] - a.lo_x) * a.inv_dx, ty = (a.y[i] - a.lo_y) * a.inv_dy;
      if (tx < 0.0 || ty < 0.0 || tx >= (double)a.nx || ty >= (double)a.ny) bin = -2;
      else bin = min((int)tx, a.nx - 1) + a.nx * min((int)ty, a.ny - 1);
    }
    const double v[kDiagVals] = {w, w * o[0], w * o[1], w * o[2], 1.0};
    if (bin >= 0) {
#pragma unroll
      for (int k = 0; k < kDiagVals; ++k) atomicAdd(&s_h[kDiagVals * bin + k], v[k]);
    }
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) tot[k].add(v[k]);
    if (bin == -1) tot[kDiagVals].add(w);
    if (bin == -2) tot[kDiagVals + 1].add(w);
  }
  // block totals: per-thread compensated values, summed in thread order
  for (int k = 0; k < kDiagVals + 2; ++k) {
    __syncthreads();
    s_red[threadIdx.x] = tot[k].value();
    __syncthreads();
    if (threadIdx.x == 0) {
      Neumaier b;
      for (int t = 0; t < (int)blockDim.x; ++t) b.add(s_red[t]);
      s_h[kDiagVals * nb + k] = b.value();
    }
  }
  __syncthreads();
  double* out = a.partial + (size_t)blockIdx.x * a.len;
  for (int k = threadIdx.x; k < a.len; k += blockDim.x) out[k] = s_h[k];
}

__global__ void k_diag_final(const double* partial, int grid, int len, double* out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < len; k += gridDim.x * blockDim.x) {
    Neumaier s;
    for (int b = 0; b < grid; ++b) s.add(partial[(size_t)b * len + k]);
    out[k] = s.value();
  }
}

}  // namespace qedk

using namespace qedk;

extern "C" qed_status qed_diag(qed_ctx* c, const qed_particles* set, const qed_diag_spec* spec, double* dev_out,
                               void* stream) {
  const qedk::NvtxRange nvtx_range("qed_diag");
  if (!c || !c->alive) {
    set_error("qed_diag: invalid context");
    return QED_ERR_NOT_INITIALIZED;
  }
  if (!set || !spec || !dev_out) {
    set_error("qed_diag: NULL argument");
    return QED_ERR_INVALID_ARG;
  }
  if (set->ctx != c) {
    set_error("qed_diag: particle set belongs to another context");
    return QED_ERR_INVALID_ARG;
  }
  const int nb = spec->nx * spec->ny;
  if (spec->nx < 1 || spec->ny < 1 || nb > kDiagMaxBins) {
    set_error("qed_diag: nx * ny must be in [1, %d]", kDiagMaxBins);
    return QED_ERR_INVALID_ARG;
  }
  DiagArgs a;
  memset(&a, 0, sizeof(a));
  if (spec->kind == QED_DIAG_SPECTRUM) {
    if (spec->ny != 1 || !(spec->lo_x > 0.0) || !(spec->hi_x > spec->lo_x) || !std::isfinite(spec->hi_x)) {
      set_error("qed_diag: spectrum needs ny = 1 and 0 < lo_x < hi_x");
      return QED_ERR_INVALID_ARG;
    }
    a.lnlo = std::log(spec->lo_x);
    a.inv_dln = spec->nx / (std::log(spec->hi_x) - a.lnlo);
  } else if (spec->kind == QED_DIAG_DETECTOR) {
    if (!(spec->hi_x > spec->lo_x) || !(spec->hi_y > spec->lo_y) || !std::isfinite(spec->hi_x - spec->lo_x) ||
        !std::isfinite(spec->hi_y - spec->lo_y)) {
      set_error("qed_diag: detector needs lo < hi on both axes");
      return QED_ERR_INVALID_ARG;
    }
    a.lo_x = spec->lo_x;
    a.lo_y = spec->lo_y;
    a.inv_dx = spec->nx / (spec->hi_x - spec->lo_x);
    a.inv_dy = spec->ny / (spec->hi_y - spec->lo_y);
  } else {
    set_error("qed_diag: unknown kind %d", spec->kind);
    return QED_ERR_INVALID_ARG;
  }
  a.kind = spec->kind;
  a.nx = spec->nx;
  a.ny = spec->ny;
  a.photon = set->species == QED_PHOTON;
  const bool zero_ref = spec->ref[0] == 0.0 && spec->ref[1] == 0.0 && spec->ref[2] == 0.0;
  a.ref[0] = zero_ref ? 1.0 : spec->ref[0];
  a.ref[1] = zero_ref ? 0.0 : spec->ref[1];
  a.ref[2] = zero_ref ? 0.0 : spec->ref[2];
  a.x = (const double*)set->soa.x; a.y = (const double*)set->soa.y; a.z = (const double*)set->soa.z;
  a.px = set->soa.px; a.py = set->soa.py; a.pz = set->soa.pz;
  a.s1 = set->soa.s1; a.s2 = set->soa.s2; a.s3 = set->soa.s3;
  a.theta = set->soa.theta; a.w = set->soa.w;
  a.n_live = &c->st->n_live[set->species];
  a.len = kDiagVals * (nb + 1) + 2;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const unsigned long long want = (set->cap + kDiagThreads - 1) / kDiagThreads;
  const int grid = (int)std::max(1ull, std::min<unsigned long long>(want, (unsigned long long)std::max(sms, 1) * 2));
  const size_t bytes = sizeof(double) * (size_t)grid * a.len;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (bytes > c->diag_bytes) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      cudaFree(c->diag_buf);
      c->diag_buf = nullptr;
      c->diag_bytes = 0;
      e = cudaMalloc(&c->diag_buf, bytes);
    }
    if (e != cudaSuccess) {
      set_error("qed_diag: scratch: %s", cudaGetErrorString(e));
      return QED_ERR_CUDA;
    }
    c->diag_bytes = bytes;
  }
  a.partial = static_cast<double*>(c->diag_buf);
  if (set->prec == QED_PREC_F64) k_diag<double><<<grid, kDiagThreads, 0, s>>>(a);
  else k_diag<float><<<grid, kDiagThreads, 0, s>>>(a);
  k_diag_final<<<(a.len + 255) / 256, 256, 0, s>>>(a.partial, grid, a.len, dev_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("qed_diag: launch failed: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  return QED_OK;
}
