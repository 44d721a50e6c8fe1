// qed_tables.cu -- builds the SF-QED lookup tables on the GPU in FP64.
//
// Every entry comes from this file's own quadrature:
//   * e^x K_nu(x) and e^x IntK_nu(x) from the integral representation
//     K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (DLMF 10.32.9), trapezoid in t;
//   * the NCS rates and inverse CDFs of the photon energy (paper Sec. III C, Eq. Wspin2
//     with W_R carrying 1/gamma) by 16-point Gauss panels in v = ln u';
//   * the NBW rates and inverse CDFs of the positron energy (Sec. III D, Eq. BW summed
//     over both spins, rho = 2/(3 chi_g delta(1-delta))) in s = logit(delta);
//   * the VB functions M_par, M_perp (Sec. III F) with the Scorer derivative
//     pi Gi'(y) = int_0^inf s exp(-s^3/3 - y s/2) cos(pi/3 + sqrt3 y s/2) ds.
// A float copy is made for the mixed-precision path.
#include <cmath>
#include <cstdio>
#include <vector>

#include "qed_common.cuh"
#include "qed_internal.h"

namespace qedk {

__constant__ double c_gl16x[16], c_gl16w[16], c_gl16b[16];

// A panel's density is carried as the logarithms of its 16 node values (in the tails it
// falls by many e-folds across one panel; its logarithm is a smooth function).
__device__ __forceinline__ double safe_log(double f) { return f > 0.0 ? log(f) : -745.0; }

// exp of the polynomial through the node logs lf[0..15], at xi in [-1,1]
__device__ double panel_dens(const double* lf, double xi) {
  double num = 0.0, den = 0.0;
  for (int j = 0; j < 16; ++j) {
    const double d = xi - c_gl16x[j];
    if (d == 0.0) return exp(lf[j]);
    const double t = c_gl16b[j] / d;
    num += t * lf[j];
    den += t;
  }
  return exp(num / den);
}

// integral of panel_dens over [xa, xb] (16-point Gauss on the sub-interval)
__device__ double panel_integral(const double* lf, double xa, double xb) {
  const double hm = 0.5 * (xb - xa), c = 0.5 * (xb + xa);
  double s = 0.0;
  for (int k = 0; k < 16; ++k) s += c_gl16w[k] * panel_dens(lf, c + hm * c_gl16x[k]);
  return s * hm;
}

// Solve for xi: mass in [-1, xi] = need (from_top = false) or mass in [xi, 1] = need
// (from_top = true); masses in panel units.  Safeguarded Newton.
__device__ double panel_solve(const double* lf, double need, bool from_top) {
  double a = -1.0, b = 1.0, xi = 0.0;
  for (int it = 0; it < 80; ++it) {
    const double g = from_top ? need - panel_integral(lf, xi, 1.0) : panel_integral(lf, -1.0, xi) - need;
    if (g > 0) b = xi; else a = xi;
    const double fx = panel_dens(lf, xi);
    double nx = fx > 0 ? xi - g / fx : 0.5 * (a + b);
    if (!(nx > a && nx < b)) nx = 0.5 * (a + b);
    if (fabs(nx - xi) < 1e-15) return nx;
    xi = nx;
  }
  return xi;
}

// ---------------------------------------------------------------------------------
// direct scaled Bessel functions
// ---------------------------------------------------------------------------------
__device__ void kdirect(double x, double& k13, double& k23, double& ik) {
  const double h = x < 64.0 ? 0.04 : 0.32 / sqrt(x);
  double a13 = 0.5, a23 = 0.5, ai = 0.5;
  for (int k = 1; k < 400000; ++k) {
    const double t = k * h;
    const double et = exp(t);
    const double ch = 0.5 * (et + 1.0 / et);
    const double arg = x * (ch - 1.0);
    if (arg > 55.0) break;
    const double e = exp(-arg);
    const double e13 = exp(t / 3.0);
    const double c13 = 0.5 * (e13 + 1.0 / e13);
    const double c23 = 2.0 * c13 * c13 - 1.0;   // cosh(2t/3)
    a13 += e * c13;
    a23 += e * c23;
    ai += e * c13 / ch;
  }
  k13 = h * a13; k23 = h * a23; ik = h * ai;
}

__global__ void k_kvalues(double* tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNK) return;
  const double hh = (kKHi - kKLo) / (kNK - 1);
  const double x = exp(kKLo + i * hh);
  double a, b, c;
  kdirect(x, a, b, c);
  tab[kOffKV + i] = a; tab[kOffKV + kNK + i] = b; tab[kOffKV + 2 * kNK + i] = c;
  // d/dlnx of the scaled functions from K13' = -K23 - K13/(3x), K23' = -K13 - 2K23/(3x),
  // IntK13' = -K13 (DLMF 10.29.2)
  tab[kOffKD + i] = x * (a - b) - a / 3.0;
  tab[kOffKD + kNK + i] = x * (b - a) - 2.0 * b / 3.0;
  tab[kOffKD + 2 * kNK + i] = x * (c - a);
}

// ---------------------------------------------------------------------------------
// NCS: density in v = ln u' (u = 1.5 chi u'), components sign sg: a + sg b
// ---------------------------------------------------------------------------------
constexpr double kV0 = -120.0, kVH = 0.5;   // panels cover ln u' in [-120, 7]
constexpr int kVP = 254;                  // panels of width 0.5
constexpr int kVN = kVP * 16;

struct Kv { double k13, k23, ik; };

__device__ __forceinline__ void ncs_dens(double chi, double up, Kv k, double& fa, double& fb) {
  const double u = 1.5 * chi * up, q = 1.0 + u, em = exp(-up);
  const double j = 1.5 * chi * up / (q * q * q);
  fa = j * em * ((2.0 + 2.0 * u + u * u) * k.k23 - q * k.ik);
  fb = j * em * u * k.k13;
}

__device__ __forceinline__ double vnode(int idx) {
  const int p = idx >> 4, k = idx & 15;
  return kV0 + (p + 0.5 * (c_gl16x[k] + 1.0)) * kVH;
}

__global__ void k_ncs_nodes(Kv* kn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > kVN) return;
  const double v = (i == kVN) ? kV0 : vnode(i);   // extra slot: the lower end v0
  Kv k;
  kdirect(exp(v), k.k13, k.k23, k.ik);
  kn[i] = k;
}

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}

__global__ void k_ncs_rates(const Kv* kn, double* tab) {
  __shared__ double sh[33];
  const int i = blockIdx.x;
  const double chi = exp(kRLo + i * ((kRHi - kRLo) / (kNR - 1)));
  double sa = 0, sb = 0;
  for (int n = threadIdx.x; n < kVN; n += blockDim.x) {
    double fa, fb;
    ncs_dens(chi, exp(vnode(n)), kn[n], fa, fb);
    sa += c_gl16w[n & 15] * fa;
    sb += c_gl16w[n & 15] * fb;
  }
  double A = block_sum(sa, sh) * 0.5 * kVH;
  double B = block_sum(sb, sh) * 0.5 * kVH;
  if (threadIdx.x == 0) {
    double fa, fb;
    ncs_dens(chi, exp(kV0), kn[kVN], fa, fb);
    A += 3.0 * fa;          // below v0 the A-density is proportional to e^{v/3}
    B += 0.6 * fb;          // and the B-density to e^{5v/3}
    tab[kOffRA + i] = A / chi;
    tab[kOffRB + i] = B / chi;
  }
  // Radiative pusher functions on the same nodes (Sec. III A, B):
  //   q = I_QED / I_C: the spin-averaged radiated power (photon energy gamma u/(1+u) times
  //   the A-density of Eq. Wspin2) over (2/3) alpha chi^2/xi_L, i.e. sqrt3/(2 pi chi^2)
  //   int du u/(1+u) [(2+2u+u^2)K23 - (1+u)IntK13]/(1+u)^3;
  //   psi1 = int du u'' K23(u'), psi3 = int du u'' K13(u'), psi2 = int du u'' IntK13(u') -
  //   psi1 with u'' = u^2/(1+u)^3 (Eq. spin1's legend).  No tail below v0 (O(u'^{4/3})).
  double s4[4] = {0.0, 0.0, 0.0, 0.0};
  for (int n = threadIdx.x; n < kVN; n += blockDim.x) {
    const double up = exp(vnode(n)), u = 1.5 * chi * up, q = 1.0 + u, em = exp(-up);
    const double wj = c_gl16w[n & 15] * 1.5 * chi * up * em * u * u / (q * q * q);
    double fa, fb;
    ncs_dens(chi, up, kn[n], fa, fb);
    s4[0] += c_gl16w[n & 15] * fa * u / q;
    s4[1] += wj * kn[n].k23;
    s4[2] += wj * kn[n].ik;
    s4[3] += wj * kn[n].k13;
  }
  double I[4];
  for (int j = 0; j < 4; ++j) I[j] = block_sum(s4[j], sh) * 0.5 * kVH;
  if (threadIdx.x == 0) {
    const double chi3 = chi * chi * chi;
    tab[kOffRR + i] = 1.7320508075688772935 / (2.0 * kPi * chi * chi) * I[0];
    tab[kOffRR + kNR + i] = I[1] / chi3;
    tab[kOffRR + 2 * kNR + i] = (I[2] - I[1]) / chi3;
    tab[kOffRR + 3 * kNR + i] = I[3] / chi3;
  }
}

// one block per (comp, chi row): node densities, panel integrals, cumulative sums,
// inversion of the cumulative integral inside a panel through its node polynomial
__global__ void k_ncs_inv(const Kv* kn, double* tab, double* scratch) {
  __shared__ double pint[kVP];
  __shared__ double lowc[kVP + 1], upc[kVP + 1];
  __shared__ double tail;
  const int comp = blockIdx.y, row = blockIdx.x;
  const double sg = comp == 0 ? -1.0 : 1.0;
  const double chi = exp(kRLo + row * ((kRHi - kRLo) / (kNCX - 1)));
  double* fn = scratch + ((size_t)comp * kNCX + row) * kVN;
  for (int n = threadIdx.x; n < kVN; n += blockDim.x) {
    double fa, fb;
    ncs_dens(chi, exp(vnode(n)), kn[n], fa, fb);
    fn[n] = fa + sg * fb;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kVP; p += blockDim.x) {
    double r = 0;
    for (int k = 0; k < 16; ++k) r += c_gl16w[k] * fn[p * 16 + k];
    pint[p] = r * 0.5 * kVH;
  }
  if (threadIdx.x == 0) {
    double fa, fb;
    ncs_dens(chi, exp(kV0), kn[kVN], fa, fb);
    tail = 3.0 * (fa + sg * fb);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    lowc[0] = tail;
    for (int p = 0; p < kVP; ++p) lowc[p + 1] = lowc[p] + pint[p];
    upc[kVP] = 0.0;
    for (int p = kVP - 1; p >= 0; --p) upc[p] = upc[p + 1] + pint[p];
  }
  for (int n = threadIdx.x; n < kVN; n += blockDim.x) fn[n] = safe_log(fn[n]);
  __syncthreads();
  const double tot = lowc[kVP];
  const double ht = (kCTHi - kCTLo) / (kNCT - 1);
  const double lnsc = log(1.5 * chi);
  for (int j = threadIdx.x; j < kNCT; j += blockDim.x) {
    const double t = kCTLo + j * ht;
    const double lev = 1.0 / (1.0 + exp(-t)), clev = 1.0 / (1.0 + exp(t));
    double v, fv;
    if (t <= 0.0 && lev * tot <= lowc[0]) {
      v = kV0 + 3.0 * log(lev * tot / lowc[0]);
      fv = lev * tot / 3.0;   // the tail integral grows as e^{v/3}
    } else {
      int p;
      double xi;
      if (t <= 0.0) {
        const double target = lev * tot;
        int lo = 0, hi = kVP;
        while (hi - lo > 1) { const int m = (lo + hi) >> 1; if (lowc[m] <= target) lo = m; else hi = m; }
        p = lo;
        xi = panel_solve(fn + p * 16, (target - lowc[p]) / (0.5 * kVH), false);
      } else {
        const double target = clev * tot;   // mass above v
        int lo = 0, hi = kVP;               // upc[lo] > target >= upc[hi]
        while (hi - lo > 1) { const int m = (lo + hi) >> 1; if (upc[m] > target) lo = m; else hi = m; }
        p = lo;
        xi = panel_solve(fn + p * 16, (target - upc[p + 1]) / (0.5 * kVH), true);
      }
      v = kV0 + (p + 0.5 * (xi + 1.0)) * kVH;
      fv = panel_dens(fn + p * 16, xi);
    }
    const size_t o = ((size_t)comp * kNCX + row) * kNCT + j;
    tab[kOffCY + o] = v + lnsc;
    tab[kOffCD + o] = lev * clev * tot / fv;
  }
}

// ---------------------------------------------------------------------------------
// NBW: delta = 1/(1+e^{-s}), s in [-16, 0]; densities scaled by exp(8/(3 chi_g))
// ---------------------------------------------------------------------------------
constexpr double kS0 = -16.0, kSH = 0.125;
constexpr int kSP = 128;
constexpr int kSN = kSP * 16;

__device__ void nbw_dens(double chig, double s, double& f0, double& f3) {
  const double d = 1.0 / (1.0 + exp(-s)), om = 1.0 / (1.0 + exp(s));
  const double dd = d * om;
  const double ex = (2.0 / (3.0 * chig)) * (1.0 - 2.0 * d) * (1.0 - 2.0 * d) / dd;
  if (ex > 740.0) { f0 = 0.0; f3 = 0.0; return; }
  double k13, k23, ik;
  kdirect(2.0 / (3.0 * chig * dd), k13, k23, ik);
  const double e = exp(-ex);
  f3 = dd * e * k23;
  f0 = dd * e * (ik + (d / om + om / d) * k23);
}

__device__ __forceinline__ double snode(int idx) {
  return kS0 + ((idx >> 4) + 0.5 * (c_gl16x[idx & 15] + 1.0)) * kSH;
}

__global__ void k_nbw(double* tab, double* scratch) {
  __shared__ double sh[33];
  __shared__ double pint[2][kSP];
  __shared__ double cum[2][kSP + 1];
  const int row = blockIdx.x;
  const double chig = exp(kBLo + row * ((kBHi - kBLo) / (kNBX - 1)));
  double* f0 = scratch + (size_t)row * 2 * kSN;
  double* f3 = f0 + kSN;
  double s0 = 0, s3 = 0;
  for (int n = threadIdx.x; n < kSN; n += blockDim.x) {
    double a, b;
    nbw_dens(chig, snode(n), a, b);
    f0[n] = a; f3[n] = b;
    s0 += c_gl16w[n & 15] * a;
    s3 += c_gl16w[n & 15] * b;
  }
  const double T0 = block_sum(s0, sh) * 0.5 * kSH;
  const double T3 = block_sum(s3, sh) * 0.5 * kSH;
  if (threadIdx.x == 0) { tab[kOffT0 + row] = 2.0 * T0; tab[kOffT3 + row] = 2.0 * T3; }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * kSP; q += blockDim.x) {
    const int comp = q / kSP, p = q % kSP;
    const double sg = comp == 0 ? -1.0 : 1.0;
    double r = 0;
    for (int k = 0; k < 16; ++k) r += c_gl16w[k] * (f0[p * 16 + k] + sg * f3[p * 16 + k]);
    pint[comp][p] = r * 0.5 * kSH;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int comp = threadIdx.x;
    cum[comp][0] = 0.0;
    for (int p = 0; p < kSP; ++p) cum[comp][p + 1] = cum[comp][p] + pint[comp][p];
  }
  __syncthreads();
  // node values of each component, written back over f0 (comp 0) and f3 (comp 1)
  for (int n = threadIdx.x; n < kSN; n += blockDim.x) {
    const double a = f0[n], b = f3[n];
    f0[n] = safe_log(a - b);
    f3[n] = safe_log(a + b);
  }
  __syncthreads();
  const double ht = (kBTHi - kBTLo) / (kNBT - 1);
  for (int q = threadIdx.x; q < 2 * kNBT; q += blockDim.x) {
    const int comp = q / kNBT, j = q % kNBT;
    const double* fc = comp == 0 ? f0 : f3;
    const double half = cum[comp][kSP];
    const double lam = exp(kBTLo + j * ht);
    double s, fs;
    if (j == kNBT - 1) {
      s = 0.0;
      fs = panel_dens(fc + (kSP - 1) * 16, 1.0);
    } else {
      const double target = lam * half;
      int lo = 0, hi = kSP;
      while (hi - lo > 1) { const int m = (lo + hi) >> 1; if (cum[comp][m] <= target) lo = m; else hi = m; }
      const double* f = fc + lo * 16;
      const double xi = panel_solve(f, (target - cum[comp][lo]) / (0.5 * kSH), false);
      s = kS0 + (lo + 0.5 * (xi + 1.0)) * kSH;
      fs = panel_dens(f, xi);
    }
    const double dl = 1.0 / (1.0 + exp(-s));
    const size_t o = ((size_t)comp * kNBX + row) * kNBT + j;
    tab[kOffBY + o] = log(dl);
    tab[kOffBD + o] = (1.0 - dl) * lam * half / fs;
  }
}

// ---------------------------------------------------------------------------------
// VB
// ---------------------------------------------------------------------------------
__device__ double pi_gi_prime(double y) {
  // pi Gi'(y), trapezoid in w = ln s over [ln(1e-9/max(1,y)), ln(1.25 min(5.6, 110/y))]
  const double smax = fmin(5.6, 110.0 / y);
  const double wa = log(1e-9) - (y > 1.0 ? log(y) : 0.0), wb = log(1.25 * smax);
  const double h = 0.03;
  const int n = (int)ceil((wb - wa) / h);
  const double r3h = 0.86602540378443864676;
  double acc = 0;
  for (int k = 0; k <= n; ++k) {
    const double s = exp(wa + k * h);
    const double term = s * s * exp(-s * s * s / 3.0 - 0.5 * y * s) * cos(kPi / 3.0 + r3h * y * s);
    acc += (k == 0 || k == n) ? 0.5 * term : term;
  }
  return acc * h;
}

// upsilon in [0, 3/4] plus 15 panels whose distance from 1 shrinks by 4 each time
// (the integrand varies on a scale ~1/chi_g next to upsilon = 1); 16-point Gauss on each.
// One thread per node: 256 threads.
__global__ void k_vb(double* tab) {
  __shared__ double sh[33];
  const int row = blockIdx.x;
  const double chig = exp(kVLo + row * ((kVHi - kVLo) / (kNV - 1)));
  double mp = 0, mq = 0;
  for (int node = threadIdx.x; node < 256; node += blockDim.x) {
    const int pnl = node >> 4, k = node & 15;
    const double a = pnl == 0 ? 0.0 : 1.0 - 0.25 * ldexp(1.0, -2 * (pnl - 1));
    const double b = 1.0 - 0.25 * ldexp(1.0, -2 * pnl);
    const double hm = 0.5 * (b - a);
    const double v = 0.5 * (a + b) + hm * c_gl16x[k], wv = hm * c_gl16w[k];
    const double omv = (1.0 - v) * (1.0 + v);
    const double x = 4.0 / (omv * chig);
    const double y = cbrt(x * x);
    const double g = y * y * pi_gi_prime(y);      // pi x^{4/3} Gi'(x^{2/3})
    mp += wv * omv * 0.5 * (1.0 + v * v / 3.0) * g;
    mq += wv * omv * (1.0 - v * v / 3.0) * g;
  }
  const double a = block_sum(mp, sh), b = block_sum(mq, sh);
  if (threadIdx.x == 0) { tab[kOffMP + row] = -11.25 * a; tab[kOffMQ + row] = -11.25 * b; }
}

__global__ void k_to_float(const double* a, float* b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Mixed path: the cubic of the 4-point Lagrange interpolant on each node interval, from the
// FP64 node values y(i-1), y(i), y(i+1), y(i+2), in powers of f = X - i (the Lagrange
// weights of nodes -1, 0, 1, 2 expanded in f), rounded to float.
__device__ void lagrange_cubic(double ym, double y0, double y1, double y2, float* c) {
  c[0] = (float)y0;
  c[1] = (float)(-ym / 3.0 - 0.5 * y0 + y1 - y2 / 6.0);
  c[2] = (float)(0.5 * ym - y0 + 0.5 * y1);
  c[3] = (float)((y2 - ym) / 6.0 + 0.5 * (y0 - y1));
}

__global__ void k_coef(const double* d, float* f) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kNV - 3) {   // VB: M_par - M_perp
    const int i = t + 1;
    double y[4];
    for (int k = 0; k < 4; ++k) y[k] = d[kOffMP + i - 1 + k] - d[kOffMQ + i - 1 + k];
    lagrange_cubic(y[0], y[1], y[2], y[3], f + kOffCoefVB + 4 * (size_t)t);
  }
  if (t < kNBX - 3) {  // NBW T0, T3
    const int i = t + 1;
    const double* a = d + kOffT0 + i - 1;
    const double* b = d + kOffT3 + i - 1;
    lagrange_cubic(a[0], a[1], a[2], a[3], f + kOffCoefT + 8 * (size_t)t);
    lagrange_cubic(b[0], b[1], b[2], b[3], f + kOffCoefT + 8 * (size_t)t + 4);
  }
  if (t < kNR - 3) {   // NCS A, B; radiative pusher q, psi1..3
    const int i = t + 1;
    const double* a = d + kOffRA + i - 1;
    const double* b = d + kOffRB + i - 1;
    lagrange_cubic(a[0], a[1], a[2], a[3], f + kOffCoefN + 8 * (size_t)t);
    lagrange_cubic(b[0], b[1], b[2], b[3], f + kOffCoefN + 8 * (size_t)t + 4);
    for (int k = 0; k < 4; ++k) {
      const double* q = d + kOffRR + (size_t)k * kNR + i - 1;
      lagrange_cubic(q[0], q[1], q[2], q[3], f + kOffCoefRR + 16 * (size_t)t + 4 * k);
    }
  }
}

// Gauss-Legendre nodes on [-1,1] by Newton iteration on P_n (host)
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 200; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

#define QCHK(call)                                                                 \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                   \
      return QED_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)

qed_status build_tables(double* d64, float* d32, cudaStream_t st) {
  double x16[16], w16[16], b16[16];
  gauss_legendre(16, x16, w16);
  for (int j = 0; j < 16; ++j) {
    double p = 1.0;
    for (int k = 0; k < 16; ++k)
      if (k != j) p *= (x16[j] - x16[k]);
    b16[j] = 1.0 / p;
  }
  QCHK(cudaMemcpyToSymbolAsync(c_gl16x, x16, sizeof(x16), 0, cudaMemcpyHostToDevice, st));
  QCHK(cudaMemcpyToSymbolAsync(c_gl16w, w16, sizeof(w16), 0, cudaMemcpyHostToDevice, st));
  QCHK(cudaMemcpyToSymbolAsync(c_gl16b, b16, sizeof(b16), 0, cudaMemcpyHostToDevice, st));
  Kv* kn = nullptr;
  double* scratch = nullptr;
  QCHK(cudaMalloc(&kn, sizeof(Kv) * (kVN + 1)));
  const size_t ncs_scr = (size_t)2 * kNCX * kVN, nbw_scr = (size_t)kNBX * 2 * kSN;
  QCHK(cudaMalloc(&scratch, sizeof(double) * (ncs_scr > nbw_scr ? ncs_scr : nbw_scr)));
  k_kvalues<<<(kNK + 127) / 128, 128, 0, st>>>(d64);
  k_ncs_nodes<<<(kVN + 1 + 127) / 128, 128, 0, st>>>(kn);
  k_ncs_rates<<<kNR, 256, 0, st>>>(kn, d64);
  k_ncs_inv<<<dim3(kNCX, 2), 256, 0, st>>>(kn, d64, scratch);
  k_nbw<<<kNBX, 256, 0, st>>>(d64, scratch);
  k_vb<<<kNV, 256, 0, st>>>(d64);
  k_to_float<<<256, 256, 0, st>>>(d64, d32, kTableLen);
  k_coef<<<(kNV + 255) / 256, 256, 0, st>>>(d64, d32);
  QCHK(cudaGetLastError());
  QCHK(cudaStreamSynchronize(st));
  QCHK(cudaFree(kn));
  QCHK(cudaFree(scratch));
  return QED_OK;
}

// ---- generator check (qed_philox_blocks) --------------------------------------------
struct PhiloxKeys { unsigned int rk[20]; };

__global__ void k_philox_blocks(const uint32_t* __restrict__ ctr, uint64_t key, uint32_t* __restrict__ out,
                                uint64_t n, const __grid_constant__ PhiloxKeys ks) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c0 = ctr[4 * i], c1 = ctr[4 * i + 1], c2 = ctr[4 * i + 2], c3 = ctr[4 * i + 3];
    const U4 a = philox10(c0, c1, c2, c3, (uint32_t)key, (uint32_t)(key >> 32));
    const U4 b = philox10_rk(c0, c1, c2, c3, ks.rk);
    uint32_t* o = out + 8 * i;
    o[0] = a.a; o[1] = a.b; o[2] = a.c; o[3] = a.d;
    o[4] = b.a; o[5] = b.b; o[6] = b.c; o[7] = b.d;
  }
}

cudaError_t launch_philox_blocks(const uint32_t* ctr, uint64_t key, uint32_t* out, uint64_t n, cudaStream_t s) {
  PhiloxKeys ks;
  philox_key_schedule(key, ks.rk);
  const uint64_t blocks = (n + 255) / 256;
  k_philox_blocks<<<(unsigned int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(ctr, key, out, n, ks);
  return cudaGetLastError();
}

}  // namespace qedk
