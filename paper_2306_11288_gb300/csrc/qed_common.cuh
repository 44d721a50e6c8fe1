// qed_common.cuh -- device-side building blocks of the GB300 SF-QED step:
// physical constants, table geometry, Philox4x32-10, small vector algebra and the
// table interpolation rules.  Written for sm_103a; precision-generic (R = double for
// the FP64 path, float for the mixed path).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qed.h"

namespace qedk {

// ---- constants (CODATA 2018; lambda = 1 um) -----------------------------------
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 2.0 * kPi;
constexpr double kAlpha = 7.2973525693e-3;
constexpr double kXiL = 2.42631023867e-6;     // hbar omega0 / (m c^2)
// classical electron radius (CODATA 2018, 2.8179403262e-15 m) in units of 1/k0 = 1 um / (2 pi)
constexpr double kR0n = 2.8179403262e-9 * 6.283185307179586477;
// medium tables (bremsstrahlung, Bethe-Heitler pairs): kNmg rows at ln E uniform on
// [ln 2, ln 2e6], kNms cumulative nodes per row; then the row totals as floats
constexpr int kNmg = 256;
constexpr int kNms = 512;
constexpr double kMgLo = 0.69314718055994531;    // ln 2
constexpr double kMgHi = 14.508657738524219;     // ln 2e6
constexpr size_t kMedBytes = 2 * (size_t)kNmg * kNms * sizeof(double) + 2 * kNmg * sizeof(float);
constexpr double kAe = 1.15965218128e-3;      // g/2 - 1
constexpr double kChiMin = 1e-4, kChiMax = 1e3;
constexpr double kChigMin = 1e-2, kChigMax = 1e3;
constexpr double kVbMin = 1e-3, kVbMax = 1e3;

// ---- table geometry (uniform grids in ln of the argument) -----------------------
constexpr int kNK = 1024;     // scaled K13, K23, IntK13 on ln x in [ln 1e-3, ln 1e5]
constexpr double kKLo = -6.907755278982137, kKHi = 11.512925464970229;
constexpr int kNR = 512;      // NCS rates A/chi, B/chi on ln chi in [ln 1e-4, ln 1e3]
constexpr double kRLo = -9.210340371976182, kRHi = 6.907755278982137;
constexpr int kNCX = 256, kNCT = 512;   // NCS inverse CDF: ln chi x logit level in [-38, 38]
constexpr double kCTLo = -38.0, kCTHi = 38.0;
constexpr int kNBX = 256, kNBT = 256;   // NBW rates / half inverse CDF: ln chi_g x ln level
constexpr double kBLo = -4.605170185988091, kBHi = 6.907755278982137;
constexpr double kBTLo = -38.0, kBTHi = 0.0;
constexpr int kNV = 1024;     // VB M_par, M_perp on ln chi_g in [ln 1e-3, ln 1e3]
constexpr double kVLo = -6.907755278982137, kVHi = 6.907755278982137;

// element offsets inside one table block (same layout in double and float copies)
constexpr size_t kOffKV = 0;                                   // [3][kNK] values
constexpr size_t kOffKD = kOffKV + 3 * kNK;                    // [3][kNK] d/dlnx
constexpr size_t kOffRA = kOffKD + 3 * kNK;                    // [kNR]
constexpr size_t kOffRB = kOffRA + kNR;
constexpr size_t kOffT0 = kOffRB + kNR;                        // [kNBX]
constexpr size_t kOffT3 = kOffT0 + kNBX;
constexpr size_t kOffMP = kOffT3 + kNBX;                       // [kNV]
constexpr size_t kOffMQ = kOffMP + kNV;
constexpr size_t kOffCY = kOffMQ + kNV;                        // [2][kNCX][kNCT]
constexpr size_t kOffCD = kOffCY + 2 * (size_t)kNCX * kNCT;
constexpr size_t kOffBY = kOffCD + 2 * (size_t)kNCX * kNCT;    // [2][kNBX][kNBT]
constexpr size_t kOffBD = kOffBY + 2 * (size_t)kNBX * kNBT;
constexpr size_t kOffRR = kOffBD + 2 * (size_t)kNBX * kNBT;    // [4][kNR] q, psi1..3 / chi^3
constexpr size_t kTableLen = kOffRR + 4 * (size_t)kNR;
// the 1-D rate tables are contiguous [kOffRA, kOffCY): staged to shared memory (FP64 path)
constexpr size_t kSmemRateLen = kOffCY - kOffRA;

// Mixed path: the same 4-point Lagrange interpolation of the 1-D rate tables, held as the
// cubic of each interval: for the row r = i - 1 of node interval i (i in [1, n-3], the
// intervals lagrange4 selects) four floats c0..c3 with p(f) = c0 + f (c1 + f (c2 + f c3)),
// f = X - i.  One 16-byte load and three FMAs per table instead of four loads, the weights
// and four FMAs.  Appended to the float copy of the tables (16-byte aligned):
//   VB:  the difference M_par - M_perp (the only combination the photon pass uses), [kNV-3][4];
//   NBW: T0 and T3 of one interval side by side, [kNBX-3][2][4];
//   NCS: A and B of one interval side by side, [kNR-3][2][4];
//   radiative pusher: q, psi1..3 / chi^3 of one interval side by side, [kNR-3][4][4]
//   (read through L1/L2, not staged).
constexpr size_t kOffCoefVB = (kTableLen + 3) / 4 * 4;
constexpr size_t kOffCoefT = kOffCoefVB + 4 * (size_t)(kNV - 3);
constexpr size_t kOffCoefN = kOffCoefT + 8 * (size_t)(kNBX - 3);
constexpr size_t kOffCoefRR = kOffCoefN + 8 * (size_t)(kNR - 3);
constexpr size_t kTab32Len = kOffCoefRR + 16 * (size_t)(kNR - 3);
// staged to shared memory by the photon pass (VB and NBW) and by the lepton pass (NCS)
constexpr size_t kCoefPhLen = kOffCoefN - kOffCoefVB;
constexpr size_t kCoefLepLen = kOffCoefRR - kOffCoefN;
static_assert(kOffCoefVB % 4 == 0 && kOffCoefT % 4 == 0 && kOffCoefN % 4 == 0 && kOffCoefRR % 4 == 0,
              "the interval cubics are read as float4");

// ---- Philox4x32-10 (Salmon et al., SC'11) ------------------------------------------
struct U4 { uint32_t a, b, c, d; };

// round multipliers and key increments (the generator's published constants)
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += kPhiloxW0; k1 += kPhiloxW1;
  }
  return U4{c0, c1, c2, c3};
}
// The same rounds with the key schedule given: rk[2r], rk[2r+1] are the two key words of
// round r (k0 + r W0, k1 + r W1 mod 2^32).  A schedule in kernel-parameter space enters
// each round as an operand, so a draw costs no key arithmetic.
__device__ __forceinline__ U4 philox10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r], n2 = hi0 ^ c3 ^ rk[2 * r + 1];
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

// two 53-bit uniforms in [0,1): counter (id_lo, id_hi, step, ctr), key = seed
struct Uni2 { double u0, u1; };
__device__ __forceinline__ Uni2 uniforms(uint64_t seed, uint64_t id, uint32_t step, uint32_t ctr) {
  U4 o = philox10((uint32_t)id, (uint32_t)(id >> 32), step, ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double s = 1.1102230246251565404e-16;  // 2^-53
  Uni2 r;
  r.u0 = (double)((((uint64_t)(o.a >> 5)) << 26) | (uint64_t)(o.b >> 6)) * s;
  r.u1 = (double)((((uint64_t)(o.c >> 5)) << 26) | (uint64_t)(o.d >> 6)) * s;
  return r;
}

// ---- vectors --------------------------------------------------------------------
template <typename R> struct V3 { R x, y, z; };
template <typename R> __device__ __forceinline__ V3<R> mk(R a, R b, R c) { return V3<R>{a, b, c}; }
template <typename R> __device__ __forceinline__ R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename R> __device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b) {
  return V3<R>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename R> __device__ __forceinline__ V3<R> operator+(V3<R> a, V3<R> b) { return V3<R>{a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename R> __device__ __forceinline__ V3<R> operator-(V3<R> a, V3<R> b) { return V3<R>{a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename R> __device__ __forceinline__ V3<R> operator*(R s, V3<R> a) { return V3<R>{s * a.x, s * a.y, s * a.z}; }
template <typename R> __device__ __forceinline__ R norm(V3<R> a) { return sqrt(dot(a, a)); }

// ---- math wrappers that pick the precision ---------------------------------------------
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float m_pow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double m_atan(double x) { return atan(x); }
__device__ __forceinline__ float m_atan(float x) { return atanf(x); }
__device__ __forceinline__ void m_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void m_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }

// ---- fast forms for the FP32 path ------------------------------------------------------
// The mixed path's tolerance (2e-5 per particle) allows the hardware approximations:
// reciprocal and reciprocal square root, exp2/log2-based exp and log, sin/cos after an
// explicit reduction to [-pi, pi], and a polynomial arctangent.  For R = double every
// helper is the ordinary accurate function, so the FP64 path is unchanged.
__device__ __forceinline__ float f_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double f_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float f_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double f_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float f_exp(float x) { return __expf(x); }
__device__ __forceinline__ double f_exp(double x) { return exp(x); }
__device__ __forceinline__ float f_log(float x) { return __logf(x); }
__device__ __forceinline__ double f_log(double x) { return log(x); }
__device__ __forceinline__ void f_sincos(float x, float* s, float* c) {
  // x - 2 pi k in two parts (6.28125 is exact in float), then the hardware sin/cos
  const float k = rintf(x * 0.15915494309189535f);
  const float r = fmaf(-k, 1.9353071795864769e-3f, fmaf(-k, 6.28125f, x));
  __sincosf(r, s, c);
}
__device__ __forceinline__ void f_sincos(double x, double* s, double* c) { sincos(x, s, c); }
// the same for an argument already in [-pi, pi] (no reduction)
__device__ __forceinline__ void f_sincos_pi(float x, float* s, float* c) { __sincosf(x, s, c); }
__device__ __forceinline__ void f_sincos_pi(double x, double* s, double* c) { sincos(x, s, c); }
// arctangent on [0,1]: odd polynomial of degree 15 fitted to atan (max error 4e-8)
__device__ __forceinline__ float atan01(float t) {
  const float t2 = t * t;
  float p = -0.004071014306f;
  p = fmaf(p, t2, 0.02193351733f);
  p = fmaf(p, t2, -0.05603502029f);
  p = fmaf(p, t2, 0.09653253829f);
  p = fmaf(p, t2, -0.1391409575f);
  p = fmaf(p, t2, 0.1994800309f);
  p = fmaf(p, t2, -0.3333003743f);
  p = fmaf(p, t2, 0.9999994061f);
  return p * t;
}
__device__ __forceinline__ float f_atan(float x) {
  const float a = fabsf(x);
  const float r = a <= 1.0f ? atan01(a) : 1.5707963267948966f - atan01(__fdividef(1.0f, a));
  return copysignf(r, x);
}
__device__ __forceinline__ double f_atan(double x) { return atan(x); }
__device__ __forceinline__ float f_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  if (mx == 0.0f) return 0.0f;
  float r = atan01(__fdividef(mn, mx));
  if (ay > ax) r = 1.5707963267948966f - r;
  if (x < 0.0f) r = 3.141592653589793f - r;
  return copysignf(r, y);
}
__device__ __forceinline__ double f_atan2(double y, double x) { return atan2(y, x); }

// ---- interpolation rules (shared specification with the test oracle) -----------------
// 4-point Lagrange on a uniform grid, X in grid units, clamped; nodes i-1..i+2 with
// i = clamp(floor(X), 1, n-3).
template <typename R>
__device__ __forceinline__ R lagrange4(const R* y, int n, R X) {
  X = X < R(0) ? R(0) : (X > R(n - 1) ? R(n - 1) : X);
  int i = (int)m_floor(X);
  i = i < 1 ? 1 : (i > n - 3 ? n - 3 : i);
  const R f = X - R(i);
  const R fm1 = f - R(1), fm2 = f - R(2), fp1 = f + R(1);
  const R wm = -f * fm1 * fm2 * R(1.0 / 6.0);
  const R w0 = fp1 * fm1 * fm2 * R(0.5);
  const R w1 = -fp1 * f * fm2 * R(0.5);
  const R w2 = fp1 * f * fm1 * R(1.0 / 6.0);
  return wm * y[i - 1] + w0 * y[i] + w1 * y[i + 1] + w2 * y[i + 2];
}

// cubic Hermite between nodes i, i+1 with derivatives (per unit of the grid variable)
template <typename R>
__device__ __forceinline__ R hermite(const R* y, const R* d, int n, R T, R h) {
  T = T < R(0) ? R(0) : (T > R(n - 1) ? R(n - 1) : T);
  int i = (int)m_floor(T);
  i = i < 0 ? 0 : (i > n - 2 ? n - 2 : i);
  const R f = T - R(i), f2 = f * f, f3 = f2 * f;
  return (R(2) * f3 - R(3) * f2 + R(1)) * __ldg(y + i) + (f3 - R(2) * f2 + f) * h * __ldg(d + i) +
         (R(3) * f2 - R(2) * f3) * __ldg(y + i + 1) + (f3 - f2) * h * __ldg(d + i + 1);
}

// 2-D: Lagrange across rows (ln chi), Hermite along the level variable
template <typename R>
__device__ __forceinline__ R table2d(const R* Y, const R* D, int nx, int nt, R X, R T, R ht) {
  X = X < R(0) ? R(0) : (X > R(nx - 1) ? R(nx - 1) : X);
  int i = (int)m_floor(X);
  i = i < 1 ? 1 : (i > nx - 3 ? nx - 3 : i);
  const R f = X - R(i);
  const R fm1 = f - R(1), fm2 = f - R(2), fp1 = f + R(1);
  const R w[4] = {-f * fm1 * fm2 * R(1.0 / 6.0), fp1 * fm1 * fm2 * R(0.5), -fp1 * f * fm2 * R(0.5),
                  fp1 * f * fm1 * R(1.0 / 6.0)};
  R acc = R(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const size_t row = (size_t)(i - 1 + k) * nt;
    acc += w[k] * hermite(Y + row, D + row, nt, T, ht);
  }
  return acc;
}

// scaled K functions e^x {K13, K23, IntK13}(x): table in [1e-3, 1e5], the two-term
// power series of I_{+-nu} below, the leading asymptote sqrt(pi/2x) above.
template <typename R>
__device__ __forceinline__ void kfun(const R* tab, R x, R& k13, R& k23, R& ik) {
  if (x < R(1e-3)) {
    const R g13 = R(2.678938534707747633), g23 = R(1.354117939426400417);
    const R g43 = g13 / R(3), g53 = R(2) * g23 / R(3), g73 = R(4) * g43 / R(3), g83 = R(5) * g53 / R(3);
    const R c = R(kPi / 1.7320508075688772935);  // pi / (2 sin(pi/3))
    const R h = R(0.5) * x, h2 = h * h;
    const R hp13 = m_pow(h, R(1.0 / 3.0)), hm13 = R(1) / hp13;
    const R hp23 = hp13 * hp13, hm23 = hm13 * hm13;
    const R e = m_exp(x);
    k13 = e * c * (hm13 * (R(1) / g23 + h2 / g53) - hp13 * (R(1) / g43 + h2 / g73));
    k23 = e * c * (hm23 * (R(1) / g13 + h2 / g43) - hp23 * (R(1) / g53 + h2 / g83));
    // int_0^x K13 = c [3 h^{2/3}/G(2/3) + (3/4) h^{8/3}/G(5/3) - (3/2) h^{4/3}/G(4/3) - (3/5) h^{10/3}/G(7/3)]
    const R h43 = hp23 * hp23;
    const R in = c * (R(3) * hp23 / g23 + R(0.75) * hp23 * h2 / g53 - R(1.5) * h43 / g43 - R(0.6) * h43 * h2 / g73);
    ik = e * (R(1.8137993642342178505) - in);   // pi/sqrt(3)
    return;
  }
  if (x > R(1e5)) {
    const R v = sqrt(R(kPi) / (R(2) * x));
    k13 = k23 = ik = v;
    return;
  }
  const R h = R((kKHi - kKLo) / (kNK - 1));
  R X = (m_log(x) - R(kKLo)) / h;
  int i = (int)m_floor(X);
  i = i < 0 ? 0 : (i > kNK - 2 ? kNK - 2 : i);
  const R f = X - R(i), f2 = f * f, f3 = f2 * f;
  const R h00 = R(2) * f3 - R(3) * f2 + R(1), h10 = (f3 - R(2) * f2 + f) * h, h01 = R(3) * f2 - R(2) * f3,
          h11 = (f3 - f2) * h;
  const R* v = tab + kOffKV;
  const R* d = tab + kOffKD;
  k13 = h00 * __ldg(v + i) + h10 * __ldg(d + i) + h01 * __ldg(v + i + 1) + h11 * __ldg(d + i + 1);
  k23 = h00 * __ldg(v + kNK + i) + h10 * __ldg(d + kNK + i) + h01 * __ldg(v + kNK + i + 1) + h11 * __ldg(d + kNK + i + 1);
  ik = h00 * __ldg(v + 2 * kNK + i) + h10 * __ldg(d + 2 * kNK + i) + h01 * __ldg(v + 2 * kNK + i + 1) +
       h11 * __ldg(d + 2 * kNK + i + 1);
}

// ---- device status -----------------------------------------------------------------
struct DevState {
  unsigned long long n_live[3];      // e-, e+, photon live counts (authoritative)
  unsigned long long next_id;
  unsigned long long n_surv;         // this step: photons surviving NBW
  unsigned long long n_nbw;          // this step: pairs created (ranked decays)
  unsigned long long n_ncs_tot;      // this step: ranked emissions
  unsigned long long n_hlow;         // this step: decayed photon slots below n_surv
  unsigned long long n_ncs_e;        // this step: ranked emissions of e- (they rank first)
  // this step, sharded (qed_step_end): added to the ids of pairs, of e- and of e+
  // emissions, and to the id counter, so that the births of all ranks are numbered as one
  // pass over the ranks in order; zero otherwise
  unsigned long long id_add[4];
  unsigned long long cursor[2];      // this step: entries written to the NBW / NCS logs
  unsigned long long ev[8];          // this step: ncs_e, ncs_p, coarse (P > 0.1), range, drop, brems e-,
                                     // brems e+, Bethe-Heitler pairs
  unsigned int done;                 // finished-block counter of the last kernel
  unsigned int epoch;                // stamp of this step's log entries
  unsigned int status;               // QED_STATUS_* bits (sticky)
  unsigned long long processed;      // particle-steps of all ensembles stepped with this state (sticky)
  // batched steps: the ensemble's clock, advanced on the device by every step
  double t;
  unsigned int step;
  float t_rel, t_mod;                // float(t - phi0), float(t mod 2 pi)
};

}  // namespace qedk
