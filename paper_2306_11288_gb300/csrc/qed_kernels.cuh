#pragma once
// qed_kernels.cuh -- the per-step kernels of the spin/polarization-resolved SF-QED hot path
// (Wan et al., arXiv:2306.11288, Secs. II-IV) for sm_103a.
//
// One step = four launches.  Caller's stream: k_photon, then (after joining the side
// stream) k_scan (two blocks: photon tiles, lepton tiles) and k_events; the context's side
// stream runs k_lepton concurrently with the photon pass.  The event kernel is a
// programmatic dependent of the scans: it samples each thread's first event while they run
// and waits for their ranks only before the births.
//   k_photon   : streaming pass over photons -- gather, Stokes frame rotation (Eq. rotation),
//                VB phase (Eq. rotation2), NBW decision (Sec. III D); photons are updated in
//                place and every decay is logged (tile, rank inside the tile) in an event log.
//   k_lepton   : streaming pass over e- then e+ -- gather, Boris (Eqs. boris1-6), T-BMT
//                (Eqs. bmt-boris1-4), x update, chi_e, NCS decision; the no-emission spin
//                update and collapse is done here; emissions are logged.
//   k_scan     : exclusive scans of the per-tile event counts (one block per scan): the
//                rank of an event is the prefix of its tile plus its rank inside the tile,
//                which orders events by particle index exactly as a sequential pass would;
//                the photon scan also lists the decayed slots (holes) in index order.
//   k_events   : one thread per task: a logged emission (photon energy, recoil, spin
//                collapse, photon Stokes, photon birth), a logged decay (pair energy, spins,
//                birth of e- and e+) or the refill of a decayed photon slot; its last block
//                closes the step (counts, ids).
// The streaming passes carry no cross-block waits; the rare events run at full warp width.
//
// GB300's FP64 pipe (and every FP32<->FP64 conversion, which runs on it) is ~70x slower
// than FP32.  The mixed path therefore touches it only for the three position additions;
// double<->float conversions of positions are done with integer bit operations.
//
// Every kernel is a template on <precision, kB (batched), ...>: qed_step.cu instantiates
// the single-ensemble kernels, qed_batch.cu the batched ones.
#include <type_traits>

#include "qed_common.cuh"
#include "qed_internal.h"
#include "qed_mlp.cuh"

namespace qedk {

// ---- double <-> float without the FP64 pipe -------------------------------------------
// double -> float by truncating the mantissa (error below one float ulp); |x| < 2^-126
// flushes to zero.  Positions never approach the float overflow threshold.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  // (hi << 3 | lo >> 29) holds the low 9 bits of the exponent E above the top 23 mantissa
  // bits.  E - (1023 - 127) is the float exponent; 1023 - 127 = 896 = 384 (mod 512), and
  // subtracting 384 << 23 (adding 2^30 mod 2^32) turns E mod 512 into E - 896 whether or
  // not E mod 512 wrapped, for float exponents 1..255.
  const unsigned int f = __funnelshift_l(lo, hi, 3) + 0x40000000u;
  const unsigned int sign = hi & 0x80000000u;
  // E < 897 (|x| < 2^-126, zero included): signed zero
  return __uint_as_float((hi << 1) >= (897u << 21) ? (f & 0x7FFFFFFFu) | sign : sign);
}
// float -> double, exact for normal floats (zero and subnormal floats give signed zero)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xFFu;
  const unsigned int hi = (b & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((b & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)(e ? hi : (b & 0x80000000u)), (int)(e ? (b << 29) : 0u));
}

// ---- external fields (paper Sec. II D) ---------------------------------------------
template <typename R>
struct EB { V3<R> E, B; };

// node index on a grid axis of n nodes: wrapped (periodic grid) or -1 outside the grid
__device__ __forceinline__ int grid_node(int i, int n, int periodic) {
  if (periodic) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return (i < 0 || i >= n) ? -1 : i;
}

template <typename R>
__device__ __forceinline__ R tsc_gather(const float* g, int nx, int ny, int periodic, double X, double Y) {
  const double fx = floor(X + 0.5), fy = floor(Y + 0.5);
  const int ig = (int)fx, jg = (int)fy;
  const R dx = (R)(X - fx), dy = (R)(Y - fy);
  const R wx[3] = {R(0.5) * (R(0.5) - dx) * (R(0.5) - dx), R(0.75) - dx * dx, R(0.5) * (R(0.5) + dx) * (R(0.5) + dx)};
  const R wy[3] = {R(0.5) * (R(0.5) - dy) * (R(0.5) - dy), R(0.75) - dy * dy, R(0.5) * (R(0.5) + dy) * (R(0.5) + dy)};
  R acc = R(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int j = grid_node(jg - 1 + b, ny, periodic);
    if (j < 0) continue;
    R row = R(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int i = grid_node(ig - 1 + c, nx, periodic);
      if (i < 0) continue;
      row += wx[c] * (R)__ldg(g + (size_t)j * nx + i);
    }
    acc += wy[b] * row;
  }
  return acc;
}

// Mixed path: the same TSC gather without FP64 arithmetic.  A position is carried to the
// grid as a cell coordinate X = I + a, I an integer node and a a float offset (|a| <~ 1),
// formed from the double position split into two floats by bit operations and from float
// splits of 1/dx and x0/dx: a is exact to its own float rounding (~1e-7 of a cell) however
// large X is.  (A plain float X = float(x) / dx would carry 2^-24 of X: 2.4e-4 of a cell at
// X = 4096, which next to a steep field, such as the evanescent field inside a dense slab,
// moves the gathered field by ~1e-3 of itself.)
//
// the low 29 mantissa bits of x that d2f_bits drops: x = d2f_bits(x) + d2f_lo(x), the low
// part rounded to float (integer operations and one conversion)
__device__ __forceinline__ float d2f_lo(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  const int se = (int)((hi >> 20) & 0x7FFu) - 1023 - 52 + 127;   // float exponent bits of 2^(e - 52)
  const float v = __uint2float_rn(lo & 0x1FFFFFFFu) * (se > 0 ? __int_as_float(se << 23) : 0.0f);
  return (hi & 0x80000000u) ? -v : v;
}
struct Cell {
  int I;     // integer part
  float a;   // offset from I
};
// X = (x - x0)/dx with 1/dx = ih + il and x0/dx = G + oh + ol
__device__ __forceinline__ Cell cell_of(double x, float ih, float il, int G, float oh, float ol) {
  const float xh = d2f_bits(x), xl = d2f_lo(x);
  const float fi = floorf(xh * ih);
  float a = fmaf(xh, ih, -fi);   // xh ih - fi, one rounding
  a = fmaf(xh, il, a);
  a = fmaf(xl, ih, a);
  a = (a - oh) - ol;
  return Cell{(int)fi - G, a};
}
// TSC weights on the grid shifted by `shift` cells (0: nodes, 0.5: half-cell positions) and
// the first of the three nodes
__device__ __forceinline__ int tsc_axis(Cell c, float shift, float w[3]) {
  const float t = c.a - shift;
  const float f = floorf(t + 0.5f);
  const float d = t - f;
  const float lo = 0.5f - d, hi = 0.5f + d;
  w[0] = 0.5f * lo * lo;
  w[1] = 0.75f - d * d;
  w[2] = 0.5f * hi * hi;
  return c.I + (int)f - 1;
}
// kPair: on grids with an even row length (and an 8-byte aligned component), read each
// stencil row as one aligned pair of nodes and one single node, 6 loads per component
// instead of 9.  Particles in random order within a tile touch a different cache line with
// nearly every lane, so fewer loads are fewer L1 wavefronts (lepton pass of the 3e7-electron
// grid: 1.85 -> 1.51 ms); particles sorted by cell touch few lines either way and pay for
// the extra selects (1.16 -> 1.21 ms).  The photon pass and the radiative lepton pass
// spilled registers with it, so only the plain and the depositing lepton passes use it.
template <bool kPair>
__device__ __forceinline__ float tsc_sum(const float* g, int nx, int ny, int periodic, int i0, int j0,
                                         const float* wx, const float* wy) {
  float acc = 0.0f;
  if (i0 >= 0 && j0 >= 0 && i0 + 2 < nx && j0 + 2 < ny) {   // interior: the whole stencil is on the grid
    const float* r = g + (size_t)j0 * nx + i0;
    if (kPair && (nx & 1) == 0 && (reinterpret_cast<uintptr_t>(g) & 7u) == 0) {
      // node pairs (i0, i0+1) or (i0+1, i0+2), whichever starts at an even index
      const int odd = i0 & 1;
      const float wa = odd ? wx[1] : wx[0], wb = odd ? wx[2] : wx[1], wc = odd ? wx[0] : wx[2];
      const float2* p2 = reinterpret_cast<const float2*>(r + odd);
      const float* ps = r + (odd ? 0 : 2);
      const int h = nx >> 1;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2 v = __ldg(p2 + b * h);
        acc += wy[b] * (wa * v.x + wb * v.y + wc * __ldg(ps + (size_t)b * nx));
      }
      return acc;
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      acc += wy[b] * (wx[0] * __ldg(r) + wx[1] * __ldg(r + 1) + wx[2] * __ldg(r + 2));
      r += nx;
    }
    return acc;
  }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int j = grid_node(j0 + b, ny, periodic);
    if (j < 0) continue;
    float row = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int i = grid_node(i0 + c, nx, periodic);
      if (i < 0) continue;
      row += wx[c] * __ldg(g + (size_t)j * nx + i);
    }
    acc += wy[b] * row;
  }
  return acc;
}

// ---- ensembles ------------------------------------------------------------------------
// A launch steps one ensemble (kB = false: its arguments are the launch parameters a.e0)
// or a batch of ensembles (kB = true: a.ens[e] in device memory, the clock of each in its
// DevState, advanced on the device so that one captured step can be replayed).
struct EnsTime {
  double t;
  unsigned int step;
  float t_rel, t_mod;
};
template <bool kB>
__device__ __forceinline__ const EnsArgs& ens_of(const StepArgs& a, int e) {
  if constexpr (kB) return a.ens[e];
  else return a.e0;
}
template <bool kB>
__device__ __forceinline__ EnsTime time_of(const EnsArgs& E) {
  if constexpr (kB) {
    const DevState* s = E.st;
    return EnsTime{s->t, s->step, s->t_rel, s->t_mod};
  } else {
    return EnsTime{E.t, E.step, E.ff.t_rel, E.ff.t_mod};
  }
}
// ensemble of global tile (or rank) g: the last e < n with off[e] <= g (off has n + 1
// non-decreasing entries and off[n] > g)
__device__ __forceinline__ int find_ens(const unsigned int* off, int n, unsigned int g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int m = (lo + hi + 1) >> 1;
    if (off[m] <= g) lo = m; else hi = m - 1;
  }
  return lo;
}

// The same for a g common to the whole warp (a streaming pass's tile), with two ballots
// instead of a search: the candidates 32 apart, then the 32 from there (off[0] = 0, so both
// ballots have a bit set; off is non-decreasing, so the highest set bit is the last index
// with off <= g).  n <= 1024; every lane of the warp calls it.
__device__ __forceinline__ int find_ens_warp(const unsigned int* off, int n, unsigned int g) {
  const int lane = (int)(threadIdx.x & 31u);
  const int ci = lane * 32;
  const unsigned int cb = __ballot_sync(0xffffffffu, ci < n && off[ci] <= g);
  const int c = (31 - __clz((int)cb)) * 32;
  const int fi = c + lane;
  const unsigned int fb = __ballot_sync(0xffffffffu, fi < n && off[fi] <= g);
  return c + (31 - __clz((int)fb));
}

// block-wide bounds over the threads with on = true, into shared b[]: b[0..3] = imin, imax,
// jmin, jmax of (i, j); b[4 + k] = the largest of the non-negative values m[k], k < kM (as
// int bits, which order non-negative floats); b[4 + kM] = the smallest positive of the
// non-negative value p (+inf when none is positive).  One warp reduction and one shared
// atomic per warp and bound.
template <int kM>
__device__ __forceinline__ void block_bounds(bool on, int i, int j, const float (&m)[kM], float p, int* b) {
  constexpr int kInfBits = 0x7f800000;
  if (threadIdx.x == 0) {
    b[0] = 0x7fffffff; b[1] = -0x7fffffff; b[2] = 0x7fffffff; b[3] = -0x7fffffff;
#pragma unroll
    for (int k = 0; k < kM; ++k) b[4 + k] = 0;
    b[4 + kM] = kInfBits;
  }
  __syncthreads();
  const int imin = __reduce_min_sync(0xffffffffu, on ? i : 0x7fffffff);
  const int imax = __reduce_max_sync(0xffffffffu, on ? i : -0x7fffffff);
  const int jmin = __reduce_min_sync(0xffffffffu, on ? j : 0x7fffffff);
  const int jmax = __reduce_max_sync(0xffffffffu, on ? j : -0x7fffffff);
  int mm[kM];
#pragma unroll
  for (int k = 0; k < kM; ++k) mm[k] = __reduce_max_sync(0xffffffffu, on ? __float_as_int(m[k]) : 0);
  const int pmin = __reduce_min_sync(0xffffffffu, on && p > 0.0f ? __float_as_int(p) : kInfBits);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(b, imin); atomicMax(b + 1, imax);
    atomicMin(b + 2, jmin); atomicMax(b + 3, jmax);
#pragma unroll
    for (int k = 0; k < kM; ++k) atomicMax(b + 4 + k, mm[k]);
    atomicMin(b + 4 + kM, pmin);
  }
  __syncthreads();
}
// FP64 path: the field formulas in double.  Mixed path: the phase is formed in float from
// host-reduced time offsets (t - phi0 and t mod 2 pi) plus float(z).
template <typename R, bool kPair = false>
__device__ __forceinline__ EB<R> gather(const EnsArgs& E, const EnsTime& tm, double x, double y, double z) {
  const qed_fields& f = E.f;
  EB<R> r;
  r.E = mk<R>(0, 0, 0);
  r.B = mk<R>(0, 0, 0);
  if (f.kind == QED_FIELD_UNIFORM) {
    r.E = mk<R>((R)f.E[0], (R)f.E[1], (R)f.E[2]);
    r.B = mk<R>((R)f.B[0], (R)f.B[1], (R)f.B[2]);
  } else if (f.kind == QED_FIELD_PLANE || f.kind == QED_FIELD_GAUSS) {
    R s, ph, zl = R(0), xr = R(0), yr = R(0);
    if (sizeof(R) == 8) {
      const double phi = tm.t + z;
      s = (R)((phi - f.phi0) * E.inv_len);
      ph = (R)phi;
      zl = (R)(f.zf - z);
    } else {
      const float zf = d2f_bits(z);
      s = (tm.t_rel + zf) * E.ff.inv_len;
      ph = tm.t_mod + zf;
      zl = E.ff.zf - zf;
    }
    if (s < R(0) || s > R(1)) return r;
    R sn, cs;
    f_sincos_pi(R(kPi) * s, &sn, &cs);
    R g = (sizeof(R) == 8 ? (R)f.a0 : (R)E.ff.a0) * sn * sn;
    if (f.kind == QED_FIELD_GAUSS) {
      if (sizeof(R) == 8) {
        const R r2 = (R)(x * x + y * y);
        const R zr_ = (R)(0.5 * f.w0 * f.w0);
        const R w0 = (R)f.w0;
        const R q = zl / zr_;
        const R w2 = w0 * w0 * (R(1) + q * q);
        g = g * (w0 / sqrt(w2)) * m_exp(-r2 / w2);
        ph = ph - R(0.5) * r2 * zl / (zl * zl + zr_ * zr_) + m_atan(q);
      } else {
        // division-free form: with q = zeta/zR, w0/w = (1+q^2)^{-1/2}
        xr = d2f_bits(x);
        yr = d2f_bits(y);
        const R r2 = xr * xr + yr * yr;
        const R q = zl * (R)E.ff.inv_zr;
        const R rs = f_rsqrt(R(1) + q * q);
        const R inv = rs * rs;
        g = g * rs * f_exp(-r2 * (R)E.ff.inv_w02 * inv);
        ph = ph - R(0.5) * r2 * q * (R)E.ff.inv_zr * inv + f_atan(q);
      }
    }
    R sp, cp;
    f_sincos(ph, &sp, &cp);
    r.E.x = g * cp;
    r.E.y = f.circular ? g * sp : R(0);
    r.B.x = r.E.y;
    r.B.y = -r.E.x;
  } else if (f.kind == QED_FIELD_GRID2D && sizeof(R) == 4) {
    const Cell cx = cell_of(x, E.ff.gix, E.ff.gix_lo, E.ff.gox_i, E.ff.gox, E.ff.gox_lo);
    const Cell cy = cell_of(y, E.ff.giy, E.ff.giy_lo, E.ff.goy_i, E.ff.goy, E.ff.goy_lo);
    float wx0[3], wx1[3], wy0[3], wy1[3];
    const int i0 = tsc_axis(cx, 0.0f, wx0), ih = tsc_axis(cx, 0.5f, wx1);
    const int j0 = tsc_axis(cy, 0.0f, wy0), jh = tsc_axis(cy, 0.5f, wy1);
    r.E.x = (R)tsc_sum<kPair>(f.gEx, f.nx, f.ny, f.periodic, ih, j0, wx1, wy0);
    r.E.y = (R)tsc_sum<kPair>(f.gEy, f.nx, f.ny, f.periodic, i0, jh, wx0, wy1);
    r.E.z = (R)tsc_sum<kPair>(f.gEz, f.nx, f.ny, f.periodic, i0, j0, wx0, wy0);
    r.B.x = (R)tsc_sum<kPair>(f.gBx, f.nx, f.ny, f.periodic, i0, jh, wx0, wy1);
    r.B.y = (R)tsc_sum<kPair>(f.gBy, f.nx, f.ny, f.periodic, ih, j0, wx1, wy0);
    r.B.z = (R)tsc_sum<kPair>(f.gBz, f.nx, f.ny, f.periodic, ih, jh, wx1, wy1);
  } else if (f.kind == QED_FIELD_GRID2D) {
    const double X = (x - f.x0) / f.dx, Y = (y - f.y0) / f.dy;
    r.E.x = tsc_gather<R>(f.gEx, f.nx, f.ny, f.periodic, X - 0.5, Y);
    r.E.y = tsc_gather<R>(f.gEy, f.nx, f.ny, f.periodic, X, Y - 0.5);
    r.E.z = tsc_gather<R>(f.gEz, f.nx, f.ny, f.periodic, X, Y);
    r.B.x = tsc_gather<R>(f.gBx, f.nx, f.ny, f.periodic, X, Y - 0.5);
    r.B.y = tsc_gather<R>(f.gBy, f.nx, f.ny, f.periodic, X - 0.5, Y);
    r.B.z = tsc_gather<R>(f.gBz, f.nx, f.ny, f.periodic, X - 0.5, Y - 0.5);
  }
  return r;
}

// x + d with d in the path's precision (mixed: exact float->double by bit operations)
__device__ __forceinline__ double add_pos(double x, double d) { return x + d; }
__device__ __forceinline__ double add_pos(double x, float d) { return x + f2d_bits(d); }

// canonical transverse frame of n: e1 = unit(y x n) (unit(n x x) near +-y), e2 = n x e1
template <typename R>
__device__ __forceinline__ void frame(V3<R> n, V3<R>& e1, V3<R>& e2) {
  R a = n.z, b = R(0), c = -n.x;
  R m2 = a * a + c * c;
  if (m2 < R(1e-20)) { a = R(0); b = n.z; c = -n.y; m2 = b * b + c * c; }
  const R inv = f_rsqrt(m2);
  e1 = mk<R>(a * inv, b * inv, c * inv);
  e2 = cross(n, e1);
}

// ---- uniforms in the path's precision ------------------------------------------------
// FP64: the exact 53-bit uniforms.  Mixed: the same numbers rounded to float (within one
// float ulp), built from the Philox words with 32-bit conversions only.
template <typename R>
struct URand { R u0, u1; };

// kRk: take the ensemble's precomputed key schedule (single-ensemble launches, where the
// ensemble's arguments are kernel parameters) instead of forming the keys from the seed
template <typename R, bool kRk>
__device__ __forceinline__ URand<R> urand(const EnsArgs& E, uint64_t id, uint32_t step, uint32_t ctr) {
  const uint32_t c0 = (uint32_t)id, c1 = (uint32_t)(id >> 32);
  const U4 o = kRk ? philox10_rk(c0, c1, step, ctr, E.rk)
                   : philox10(c0, c1, step, ctr, (uint32_t)E.seed, (uint32_t)(E.seed >> 32));
  URand<R> r;
  if (sizeof(R) == 8) {
    const double s = 1.1102230246251565404e-16;  // 2^-53, as in uniforms()
    r.u0 = (R)((double)((((uint64_t)(o.a >> 5)) << 26) | (uint64_t)(o.b >> 6)) * s);
    r.u1 = (R)((double)((((uint64_t)(o.c >> 5)) << 26) | (uint64_t)(o.d >> 6)) * s);
  } else {
    r.u0 = (R)(__uint2float_rn(o.a >> 5) * 0x1p-27f + __uint2float_rn(o.b >> 6) * 0x1p-53f);
    r.u1 = (R)(__uint2float_rn(o.c >> 5) * 0x1p-27f + __uint2float_rn(o.d >> 6) * 0x1p-53f);
  }
  return r;
}

// ---- table access --------------------------------------------------------------------
// Mixed path: the row of the interval lagrange4 selects for X (grid units) and the offset f
// of X in it; the cubic of one row
__device__ __forceinline__ int coef_row(float X, int n, float& f) {
  X = fminf(fmaxf(X, 0.0f), (float)(n - 1));
  int i = __float2int_rd(X);
  i = min(max(i, 1), n - 3);
  f = X - (float)i;
  return i - 1;
}
__device__ __forceinline__ float coef_cubic(float4 c, float f) { return fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x); }

template <typename R>
struct Tabs {
  const R* g;     // full table block in global memory
  const R* s;     // FP64 path: the 1-D rate tables (shared memory in the streaming kernels)
  // mixed path: the interval cubics of the VB difference, NBW and NCS rate tables (shared
  // memory where the streaming kernel staged them, else global memory)
  const float4* cv;
  const float4* cb;
  const float4* cn;
  __device__ __forceinline__ void ncs_rates(R chi, R& A, R& B) const {
    const R X = (f_log(chi) - R(kRLo)) * R((kNR - 1) / (kRHi - kRLo));
    if constexpr (sizeof(R) == 4) {
      float f;
      const int r = coef_row(X, kNR, f);
      A = chi * coef_cubic(cn[2 * r], f);
      B = chi * coef_cubic(cn[2 * r + 1], f);
    } else {
      A = chi * lagrange4(s, kNR, X);
      B = chi * lagrange4(s + kNR, kNR, X);
    }
  }
  __device__ __forceinline__ R ncs_inv(int comp, R chi, R t) const {
    const R X = (m_log(chi) - R(kRLo)) * R((kNCX - 1) / (kRHi - kRLo));
    const R ht = R((kCTHi - kCTLo) / (kNCT - 1));
    const size_t o = (size_t)comp * kNCX * kNCT;
    return table2d(g + kOffCY + o, g + kOffCD + o, kNCX, kNCT, X, (t - R(kCTLo)) / ht, ht);
  }
  __device__ __forceinline__ void nbw_rates(R chig, R& T0, R& T3) const {
    const R X = (f_log(chig) - R(kBLo)) * R((kNBX - 1) / (kBHi - kBLo));
    const R damp = f_exp(R(-8.0 / 3.0) * f_rcp(chig));
    if constexpr (sizeof(R) == 4) {
      float f;
      const int r = coef_row(X, kNBX, f);
      T0 = damp * coef_cubic(cb[2 * r], f);
      T3 = damp * coef_cubic(cb[2 * r + 1], f);
    } else {
      T0 = damp * lagrange4(s + (kOffT0 - kOffRA), kNBX, X);
      T3 = damp * lagrange4(s + (kOffT3 - kOffRA), kNBX, X);
    }
  }
  __device__ __forceinline__ R nbw_inv(int comp, R chig, R t) const {
    const R X = (m_log(chig) - R(kBLo)) * R((kNBX - 1) / (kBHi - kBLo));
    const R ht = R((kBTHi - kBTLo) / (kNBT - 1));
    const size_t o = (size_t)comp * kNBX * kNBT;
    return table2d(g + kOffBY + o, g + kOffBD + o, kNBX, kNBT, X, (t - R(kBTLo)) / ht, ht);
  }
  // M_par - M_perp (4 - 7 below the table)
  __device__ __forceinline__ R vb_md(R chig) const {
    if (chig < R(kVbMin)) return R(-3);
    const R X = (f_log(chig) - R(kVLo)) * R((kNV - 1) / (kVHi - kVLo));
    if constexpr (sizeof(R) == 4) {
      float f;
      const int r = coef_row(X, kNV, f);
      return coef_cubic(cv[r], f);
    } else {
      return lagrange4(s + (kOffMP - kOffRA), kNV, X) - lagrange4(s + (kOffMQ - kOffRA), kNV, X);
    }
  }
  __device__ __forceinline__ void k(R x, R& k13, R& k23, R& ik) const { kfun(g, x, k13, k23, ik); }
  // radiative pusher functions (read through L1/L2: used only with the radiative flags):
  // q(chi) (1 below chi_min) and psi1..3 = chi^3 times the tabulated psi/chi^3
  __device__ __forceinline__ void rr_funcs(R chi, R& qf, R& p1, R& p2, R& p3) const {
    const R X = (f_log(chi) - R(kRLo)) * R((kNR - 1) / (kRHi - kRLo));
    const R chi3 = chi * chi * chi;
    if constexpr (sizeof(R) == 4) {
      float f;
      const float4* c = reinterpret_cast<const float4*>(g + kOffCoefRR) + 4 * coef_row(X, kNR, f);
      qf = chi < R(kChiMin) ? R(1) : coef_cubic(c[0], f);
      p1 = chi3 * coef_cubic(c[1], f);
      p2 = chi3 * coef_cubic(c[2], f);
      p3 = chi3 * coef_cubic(c[3], f);
    } else {
      qf = chi < R(kChiMin) ? R(1) : lagrange4(g + kOffRR, kNR, X);
      p1 = chi3 * lagrange4(g + kOffRR + kNR, kNR, X);
      p2 = chi3 * lagrange4(g + kOffRR + 2 * kNR, kNR, X);
      p3 = chi3 * lagrange4(g + kOffRR + 3 * kNR, kNR, X);
    }
  }
};

// ---- radiative pusher (Sec. III A "Algorithms of the Radiative Pusher"; Sec. III B) ----
// Evaluated once per step at the time-centred momentum pb = (p^{n-1/2} + p_L^{n+1/2})/2 of
// the Boris step and the fields at x^n.  The LL force keeps the second and third terms of
// Eq. eq1-1 (the field-derivative term is dropped), with 1/gamma on E(p.E) as in Eq. eq1;
// its third term is written through chi: gamma p [(E + beta x B)^2 - (beta.E)^2] =
// chi^2 beta / xi_L^2.  The radiative T-BMT term -P[psi1 S + psi2 (S.beta) beta + psi3 n_B]
// (Eq. spin1), n_B = n x a_hat, is applied as two half kicks around the T-BMT rotation.
template <typename R>
struct RadSpin {
  R P, p1, p2, p3;
  V3<R> be, zeta;
  bool on;
};

template <typename R>
__device__ __forceinline__ void rad_push(const Tabs<R>& tb, uint32_t flags, R q, R dt, const EB<R>& f,
                                         const V3<R>& p0, V3<R>& pn, RadSpin<R>& rs, bool& range) {
  rs.on = false;
  const V3<R> pb = R(0.5) * (p0 + pn);
  const R pm2 = dot(pb, pb);
  const R gb2 = R(1) + pm2;
  const R inv_gb = f_rsqrt(gb2);
  const R gb = gb2 * inv_gb;
  const V3<R> be = inv_gb * pb;
  R chi = R(0), vm2 = R(0);
  V3<R> v = mk<R>(0, 0, 0), nb = mk<R>(0, 0, 0);
  if (pm2 > R(0)) {
    nb = f_rsqrt(pm2) * pb;
    const R nE = dot(nb, f.E);
    v = gb * (f.E - nE * nb) + cross(pb, f.B);
    vm2 = dot(v, v);
    if (sizeof(R) == 4) {
      // FP64 island: gamma E_perp and p x B cancel (co-propagation)
      const V3<R> a1 = gb * (f.E - nE * nb), a2 = cross(pb, f.B);
      if (vm2 < R(1e-4) * (dot(a1, a1) + dot(a2, a2))) {
        const double px = pb.x, py = pb.y, pz = pb.z;
        const double G1 = sqrt(1.0 + px * px + py * py + pz * pz), pmd = sqrt(px * px + py * py + pz * pz);
        const double nx = px / pmd, ny = py / pmd, nz = pz / pmd;
        const double Ex = f.E.x, Ey = f.E.y, Ez = f.E.z, Bx = f.B.x, By = f.B.y, Bz = f.B.z;
        const double ne = nx * Ex + ny * Ey + nz * Ez;
        const double vx = G1 * (Ex - ne * nx) + (py * Bz - pz * By);
        const double vy = G1 * (Ey - ne * ny) + (pz * Bx - px * Bz);
        const double vz = G1 * (Ez - ne * nz) + (px * By - py * Bx);
        v = mk<R>((R)vx, (R)vy, (R)vz);
        vm2 = (R)(vx * vx + vy * vy + vz * vz);
      }
    }
    const R c2 = vm2 + nE * nE;
    chi = c2 > R(0) ? R(kXiL) * c2 * f_rsqrt(c2) : R(0);
  }
  R chit = chi;
  if (chit > R(kChiMax)) { chit = R(kChiMax); range = true; }
  R qf = R(1), p1 = R(0), p2 = R(0), p3 = R(0);
  if (chit > R(0)) tb.rr_funcs(chit, qf, p1, p2, p3);
  if (flags & (QED_F_LL | QED_F_MLL)) {
    const R qq = (flags & QED_F_MLL) ? qf : R(1);
    const V3<R> ExB = cross(f.E, f.B);
    const V3<R> BxBxp = cross(f.B, cross(f.B, pb));
    const R pE = dot(pb, f.E);
    const R c2 = R(2.0 / 3.0 * kAlpha * kXiL), c3 = R(2.0 / 3.0 * kAlpha / kXiL) * chi * chi;
    const V3<R> F = qq * (c2 * (ExB + inv_gb * BxBxp + (inv_gb * pE) * f.E) - c3 * be);
    pn = pn + dt * F;
  }
  if ((flags & QED_F_MBMT) && vm2 > R(0) && chi > R(0)) {
    const V3<R> av = (q * f_rsqrt(vm2)) * v;
    rs.zeta = cross(nb, av);
    rs.P = R(kAlpha / (1.7320508075688772935 * kPi * kXiL)) * inv_gb;
    rs.p1 = p1; rs.p2 = p2; rs.p3 = p3;
    rs.be = be;
    rs.on = true;
  }
}

// S += dt/2 (dS/dt)_R
template <typename R>
__device__ __forceinline__ void rad_spin_half(const RadSpin<R>& rs, R dt, V3<R>& S) {
  const R sb = dot(S, rs.be);
  const R h = R(-0.5) * dt * rs.P;
  S = S + h * (rs.p1 * S + (rs.p2 * sb) * rs.be + rs.p3 * rs.zeta);
}

// Tables in global memory (every pointer into the table block).
template <typename R>
__device__ __forceinline__ Tabs<R> tabs_global(const void* tables) {
  const R* g = reinterpret_cast<const R*>(tables);
  Tabs<R> t{g, g + kOffRA, nullptr, nullptr, nullptr};
  if constexpr (sizeof(R) == 4) {
    t.cv = reinterpret_cast<const float4*>(g + kOffCoefVB);
    t.cb = reinterpret_cast<const float4*>(g + kOffCoefT);
    t.cn = reinterpret_cast<const float4*>(g + kOffCoefN);
  }
  return t;
}

// What a streaming kernel stages to shared memory: FP64 path, the 1-D rate tables; mixed
// path, the interval cubics it uses (photon pass: VB and NBW; lepton pass: NCS).
template <typename R, bool kPh> struct SmemTab {
  static constexpr size_t n = sizeof(R) == 8 ? kSmemRateLen : (kPh ? kCoefPhLen : kCoefLepLen);
};
// global -> shared 1-D bulk copy (TMA) of `bytes` (16-byte aligned ends, a multiple of 16),
// completing on the mbarrier bar
__device__ __forceinline__ void tma_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned int bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Copies them to s (16-byte aligned) by TMA -- one bulk copy issued by one thread, completed
// on an mbarrier that every thread waits on (bounded) -- and points the table accessors
// there.  Block size kTile; the caller synchronises the block afterwards.  A wait that
// gives up (never expected) sets QED_STATUS_TIMEOUT, waits once more for the copy in
// flight, and copies the tables with plain loads.
template <typename R, bool kPh>
__device__ __forceinline__ void stage_rates(Tabs<R>& tb, R* s, unsigned int* status) {
  constexpr size_t o = sizeof(R) == 8 ? kOffRA : (kPh ? kOffCoefVB : kOffCoefN);
  constexpr size_t kEl = 16 / sizeof(R);                       // elements per 16 bytes
  constexpr size_t n = SmemTab<R, kPh>::n;
  static_assert(o % kEl == 0 && n % kEl == 0, "16-byte table segments");
  constexpr unsigned int kBytes = (unsigned int)(n * sizeof(R));
  __shared__ __align__(8) unsigned long long s_bar;
  if (threadIdx.x == 0) {
    mlp_mbar_init(&s_bar);
    tma_expect_tx(&s_bar, kBytes);
    tma_load_1d(s, tb.g + o, kBytes, &s_bar);
  }
  __syncthreads();   // the barrier's initialisation before anyone waits on it
  if (!mlp_mbar_wait(&s_bar, 0u)) {
    if (threadIdx.x == 0) atomicOr(status, QED_STATUS_TIMEOUT);
    mlp_mbar_wait(&s_bar, 0u);
    const uint4* src = reinterpret_cast<const uint4*>(tb.g + o);
    uint4* dst = reinterpret_cast<uint4*>(s);
    for (int q = (int)threadIdx.x; q < (int)(n / kEl); q += kTile) dst[q] = src[q];
  }
  if constexpr (sizeof(R) == 8) {
    tb.s = s;
  } else if constexpr (kPh) {
    tb.cv = reinterpret_cast<const float4*>(s);
    tb.cb = reinterpret_cast<const float4*>(s + (kOffCoefT - kOffCoefVB));
  } else {
    tb.cn = reinterpret_cast<const float4*>(s);
  }
}

template <typename T>
__device__ __forceinline__ T ld(const void* p, unsigned long long i) { return reinterpret_cast<const T*>(p)[i]; }
template <typename T>
__device__ __forceinline__ void stv(void* p, unsigned long long i, T v) { reinterpret_cast<T*>(p)[i] = v; }

__device__ __forceinline__ void count_event(unsigned long long* ctr, bool flag) {
  const unsigned int b = __ballot_sync(0xffffffffu, flag);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(ctr, (unsigned long long)__popc(b));
}

// ---- event logs ------------------------------------------------------------------------
// bit 31 of NbwRec::ens / NcsRec::species: the event is a matter process (a Bethe-Heitler
// decay / a bremsstrahlung emission) rather than NBW / NCS; the rank space is shared
constexpr unsigned int kEvMedium = 0x80000000u;
template <typename R>
struct NbwRec {
  unsigned long long i;      // photon slot
  unsigned int tile, r_in;   // tile and rank inside the tile
  unsigned int stamp, ens;   // step stamp; ensemble of the photon
  double x, y, z;            // x^n (the photon itself has moved on in its slot)
  R chig, rmix, p1x, p1y, p1z;
  // the photon as the decision left it (k, Stokes after this step's rotations, weight,
  // id): the event reads none of the slot, which a refill or a birth may take meanwhile
  R kx, ky, kz, x1, x2, x3, w;
  unsigned long long id;
};
template <typename R>
struct NcsRec {
  unsigned long long i;      // lepton slot
  unsigned int tile, r_in, stamp, species;   // species: e- 0 / e+ 1, | ensemble << 1
  R chi, ax, ay, az;         // chi_e and the unit acceleration direction
};


// In-tile ranks of flagged threads and one reservation in the event log per tile.
// Returns the thread's slot in the log, or ~0 when the tile's events were not logged
// (log full: QED_STATUS_LOG_FULL; the logs are sized for one event per particle, so this
// is a safeguard).  tile_cnt[tile] receives the logged count.
struct TileShared {
  unsigned int wc[kTile / 32];
  unsigned long long base;
  int ok;
};

__device__ __forceinline__ unsigned long long tile_log(bool flag, unsigned int tile, unsigned int* tile_cnt,
                                                       unsigned long long* cursor, unsigned long long cap,
                                                       unsigned int* status, TileShared& sh, unsigned int* r_in) {
  // most tiles carry no event: one barrier settles them
  if (!__syncthreads_or(flag)) {
    if (threadIdx.x == 0) tile_cnt[tile] = 0u;
    *r_in = 0;
    return ~0ull;
  }
  const unsigned int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int ballot = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) sh.wc[warp] = __popc(ballot);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int run = 0;
    for (int w = 0; w < kTile / 32; ++w) {
      const unsigned int c = sh.wc[w];
      sh.wc[w] = run;
      run += c;
    }
    const unsigned long long base = atomicAdd(cursor, (unsigned long long)run);
    const int ok = base + run <= cap;
    if (!ok) atomicOr(status, QED_STATUS_LOG_FULL);
    sh.base = base;
    sh.ok = ok;
    tile_cnt[tile] = ok ? run : 0u;
  }
  __syncthreads();
  const unsigned int r = sh.wc[warp] + __popc(ballot & ((1u << lane) - 1u));
  *r_in = r;
  const unsigned long long slot = (flag && sh.ok) ? sh.base + r : ~0ull;
  __syncthreads();   // sh is reused by the next tile
  return slot;
}

template <typename R> struct Occ { static constexpr int v = sizeof(R) == 4 ? 4 : 2; };
// the photon pass holds a second tile's records in registers
template <typename R> struct OccPh { static constexpr int v = sizeof(R) == 4 ? 3 : 2; };

// ---- programmatic dependent launch ------------------------------------------------------
// The event kernels are launched as programmatic dependents of the kernel before them on
// the stream: they may be scheduled while it drains and wait here for its completion (and
// the visibility of its writes) before touching any data.  Without the launch attribute
// both instructions return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- matter (Sec. III E): bremsstrahlung and Bethe-Heitler pairs ----------------------
// Tables of the medium (qed_medium.cu): brems rows then pair rows, kNmg x kNms cumulative
// cross-sections (units alpha r0^2), then the row totals as floats.
__device__ __forceinline__ bool in_medium(const StepArgs& a, double x, double y, double z) {
  const double v = a.med_axis == 0 ? x : (a.med_axis == 1 ? y : z);
  return v >= a.med_lo && v < a.med_hi;
}
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
// total cross-section of process `which` (0 brems, 1 pairs) at ln E: linear in ln E between
// the rows (FP64 path: the FP64 totals; mixed path: their float copies); zero below the
// first row, clamped (and counted) above the last
template <typename R>
__device__ __forceinline__ R med_sigma(const StepArgs& a, int which, R lnE, bool& range) {
  R t = (lnE - R(kMgLo)) * R((kNmg - 1) / (kMgHi - kMgLo));
  if (!(t >= R(0))) return R(0);
  if (t > R(kNmg - 1)) {
    t = R(kNmg - 1);
    range = true;
  }
  int i = (int)t;
  i = i > kNmg - 2 ? kNmg - 2 : i;
  const R w = t - R(i);
  R s0, s1;
  if constexpr (sizeof(R) == 8) {
    const double* C = a.med_c + (size_t)which * kNmg * kNms;
    s0 = C[(size_t)i * kNms + kNms - 1];
    s1 = C[(size_t)(i + 1) * kNms + kNms - 1];
  } else {
    const float* T = a.med_tot + which * kNmg;
    s0 = __ldg(T + i);
    s1 = __ldg(T + i + 1);
  }
  return (R(1) - w) * s0 + w * s1;
}
// The energy fraction (brems y, pairs x) at energy E for a uniform r (FP64 on both paths):
// rows i, i+1 around ln E mixed linearly, the node interval whose cumulative brackets
// r sigma(E), linear inside it; s -> the fraction uniform in ln(v/(1-v)) between the end
// points at E (brems [k_min/E, 1 - 1/E], pairs [1/E, 1 - 1/E]).
static __device__ __noinline__ double med_sample(const StepArgs& a, int which, double E, double r) {
  const double* C = a.med_c + (size_t)which * kNmg * kNms;
  double t = (log(E) - kMgLo) / ((kMgHi - kMgLo) / (kNmg - 1));
  double s = 0.0;
  if (t >= 0.0) {
    if (t > kNmg - 1) t = kNmg - 1;
    int i = (int)floor(t);
    i = i > kNmg - 2 ? kNmg - 2 : i;
    const double w = t - i;
    const double* A = C + (size_t)i * kNms;
    const double* B = A + kNms;
    const double tot = (1.0 - w) * A[kNms - 1] + w * B[kNms - 1];
    if (tot > 0.0) {
      const double target = r * tot;
      int lo = 0, hi = kNms - 1;
      while (hi - lo > 1) {
        const int m = (lo + hi) / 2;
        const double cm = (1.0 - w) * A[m] + w * B[m];
        if (cm <= target) lo = m; else hi = m;
      }
      const double c0 = (1.0 - w) * A[lo] + w * B[lo], c1 = (1.0 - w) * A[lo + 1] + w * B[lo + 1];
      const double f = c1 > c0 ? (target - c0) / (c1 - c0) : 0.0;
      s = (lo + f) / (kNms - 1);
    }
  }
  const double vlo = which == 0 ? a.med_kmin / E : 1.0 / E, vhi = 1.0 - 1.0 / E;
  const double tlo = log(vlo / (1.0 - vlo)), thi = log(vhi / (1.0 - vhi));
  return 1.0 / (1.0 + exp(-(tlo + s * (thi - tlo))));
}

// ======================================================================================
// photon streaming pass
// ======================================================================================
// A photon's input record.  The pass loads the next tile's records before it computes the
// current tile (register double buffering), so the loads of one tile are in flight while
// the previous one is computed: the pass's own loads hide behind its arithmetic instead of
// stalling every warp of the block at the top of each tile.
template <typename R>
struct PhIn {
  double x, y, z;
  V3<R> k, xi;
  R th;
  uint64_t id;
};

template <typename R>
__device__ __forceinline__ void ph_load(const SpeciesArgs& P, unsigned int i, bool live, PhIn<R>& v) {
  if (live) {
    v.x = P.x[i]; v.y = P.y[i]; v.z = P.z[i];
    v.k = mk<R>(ld<R>(P.px, i), ld<R>(P.py, i), ld<R>(P.pz, i));
    v.xi = mk<R>(ld<R>(P.s1, i), ld<R>(P.s2, i), ld<R>(P.s3, i));
    v.th = ld<R>(P.theta, i);
    v.id = P.id[i];
  } else {
    v.x = 0; v.y = 0; v.z = 0;
    v.k = mk<R>(1, 0, 0);
    v.xi = mk<R>(0, 0, 0);
    v.th = 0;
    v.id = 0;
  }
}

// where a tile's photons are: ensemble, first slot of the thread, live flag
struct PhTile {
  int ens;
  unsigned int i;
  bool live;
};

template <bool kB>
__device__ __forceinline__ PhTile ph_tile(const StepArgs& a, const unsigned int* s_off, unsigned long long n_one,
                                          unsigned int tile) {
  PhTile t;
  t.ens = kB ? find_ens_warp(s_off, a.n_ens, tile) : 0;
  const EnsArgs& E = ens_of<kB>(a, t.ens);
  const SpeciesArgs& P = E.sp[2];
  const unsigned long long n = kB ? (P.present ? E.st->n_live[2] : 0ull) : n_one;
  t.i = (tile - (kB ? s_off[t.ens] : 0u)) * kTile + threadIdx.x;   // capacity <= 2^32 - 256
  t.live = t.i < (unsigned int)n;
  return t;
}

template <typename R, bool kB, bool kSm, bool kMed = false>
__global__ void __launch_bounds__(kTile, kB ? Occ<R>::v : OccPh<R>::v) k_photon(const __grid_constant__ StepArgs a) {
  // single-ensemble launches double-buffer the records in registers; batched launches
  // (whose tile-to-ensemble search needs the registers) load each tile at its top
  constexpr bool kPf = !kB;
  pdl_trigger();
  __shared__ __align__(16) R s_rates[kSm ? SmemTab<R, true>::n : 1];
  __shared__ TileShared s_tile;
  __shared__ unsigned int s_off[kB ? kMaxEns + 1 : 1];
  DevState* gst = a.st;
  unsigned int ntiles;
  unsigned long long n_one = 0;   // single ensemble: its photon count, read once
  if constexpr (kB) {
    for (int e = threadIdx.x; e <= a.n_ens; e += blockDim.x) s_off[e] = a.map->ph_tile0[e];
    ntiles = a.map->ph_tile0[a.n_ens];
  } else {
    n_one = a.e0.sp[2].present ? a.e0.st->n_live[2] : 0ull;
    ntiles = (unsigned int)((n_one + kTile - 1) / kTile);
  }
  Tabs<R> tb = tabs_global<R>(a.tables);
  if constexpr (kSm) stage_rates<R, true>(tb, s_rates, &a.st->status);
  __syncthreads();
  const unsigned int epoch = gst->epoch;
  const R dt = sizeof(R) == 8 ? (R)a.dt : (R)a.fdt;
  NbwRec<R>* evlog = reinterpret_cast<NbwRec<R>*>(a.rec[0]);
  PhTile cur{0, 0u, false};
  PhIn<R> in;
  if (kPf && blockIdx.x < ntiles) {
    cur = ph_tile<kB>(a, s_off, n_one, blockIdx.x);
    ph_load<R>(ens_of<kB>(a, cur.ens).sp[2], cur.i, cur.live, in);
  }
  for (unsigned int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    PhTile nxt{0, 0u, false};
    PhIn<R> in_n;
    if constexpr (kPf) {
      // the next tile's records, in flight while this tile is computed
      const unsigned int tile_n = tile + gridDim.x;
      if (tile_n < ntiles) nxt = ph_tile<kB>(a, s_off, n_one, tile_n);
      ph_load<R>(ens_of<kB>(a, nxt.ens).sp[2], nxt.i, nxt.live, in_n);
    } else {
      cur = ph_tile<kB>(a, s_off, n_one, tile);
      ph_load<R>(ens_of<kB>(a, cur.ens).sp[2], cur.i, cur.live, in);
    }

    const int ens = cur.ens;
    const EnsArgs& E = ens_of<kB>(a, ens);
    const EnsTime tm = time_of<kB>(E);
    DevState* st = E.st;
    const SpeciesArgs& P = E.sp[2];
    const unsigned int i = cur.i;
    const bool live = cur.live;
    const double x = in.x, y = in.y, z = in.z;
    const V3<R> k = in.k;
    V3<R> xi = in.xi;
    R th = in.th;
    const uint64_t id = in.id;
    bool decay = false, range = false;
    const R om2 = dot(k, k);
    const R inv_om = f_rsqrt(om2);
    const R om = om2 * inv_om;
    const V3<R> nn = inv_om * k;
    V3<R> P1 = mk<R>(0, 0, 0);
    R chig = 0, rmix = 0;
    if (live && (a.flags & (QED_F_VB | QED_F_NBW))) {
      const EB<R> f = gather<R>(E, tm, x, y, z);
      const R ne = dot(nn, f.E);
      const V3<R> Er = f.E - ne * nn + cross(nn, f.B);
      const R er2 = dot(Er, Er);
      if (er2 > R(0)) {
        const R inv_er = f_rsqrt(er2);
        const R er = er2 * inv_er;
        chig = R(kXiL) * om * er;
        P1 = inv_er * Er;
        // the canonical frame of n without its normalisation (atan2 needs only the ratio)
        R fa = nn.z, fb = R(0), fc = -nn.x;
        if (fa * fa + fc * fc < R(1e-20)) { fa = R(0); fb = nn.z; fc = -nn.y; }
        const V3<R> e1 = mk<R>(fa, fb, fc), e2 = cross(nn, e1);
        const R thn = f_atan2(dot(P1, e2), dot(P1, e1));
        R s2, c2;
        f_sincos(R(2) * (thn - th), &s2, &c2);
        const R x1 = xi.x * c2 - xi.z * s2, x3 = xi.x * s2 + xi.z * c2;
        xi.x = x1; xi.z = x3;
        th = thn;
        if (a.flags & QED_F_VB) {
          const R md = tb.vb_md(chig > R(kVbMax) ? R(kVbMax) : chig);
          const R dphi = md * R(kAlpha / (90.0 * kPi) * kXiL) * om * er * er * dt;
          R sd, cd;
          if (dphi < R(1e-2) && dphi > R(-1e-2)) {
            const R d2 = dphi * dphi;
            if (sizeof(R) == 8) {   // Taylor to 5th/6th order: error below 2e-15
              sd = dphi * (R(1) - d2 * (R(1.0 / 6.0) - d2 * R(1.0 / 120.0)));
              cd = R(1) - d2 * (R(0.5) - d2 * (R(1.0 / 24.0) - d2 * R(1.0 / 720.0)));
            } else {                // to 3rd/2nd order: the next terms are below 1e-9
              sd = dphi * (R(1) - d2 * R(1.0 / 6.0));
              cd = R(1) - d2 * R(0.5);
            }
          } else {
            f_sincos(dphi, &sd, &cd);
          }
          const R y1 = cd * xi.x - sd * xi.y, y2 = sd * xi.x + cd * xi.y;
          xi.x = y1; xi.y = y2;
        }
        if ((a.flags & QED_F_NBW) && om >= R(2) && chig >= R(kChigMin)) {
          if (chig > R(kChigMax)) { chig = R(kChigMax); range = true; }
          R T0, T3;
          tb.nbw_rates(chig, T0, T3);
          const R Pd = R(kAlpha / (1.7320508075688772935 * kPi * kXiL)) * inv_om * (T0 - xi.z * T3) * dt;
          const URand<R> u = urand<R, !kB>(E, id, tm.step, 3u);
          decay = u.u0 < Pd;
          // one event per photon per step is coarse where T dt > 0.1 (rare: no ballot)
          if (Pd > R(0.1)) atomicAdd(&st->ev[2], 1ull);
          rmix = u.u1;
        }
      }
    }
    bool bh = false;
    if constexpr (kMed) {
      // Bethe-Heitler pair creation in the medium, if the photon did not decay by NBW:
      // P = 1 - exp(-n sigma(k) c dt) (Sec. III E)
      if (live && !decay && (a.flags & QED_F_BH) && om > R(2) && in_medium(a, x, y, z)) {
        const R sig = med_sigma<R>(a, 1, f_log(om), range);
        const R Pb = -m_expm1(-R(a.med_nar2) * sig * dt);
        const URand<R> u = urand<R, !kB>(E, id, tm.step, 6u);
        if (Pb > R(0.1)) atomicAdd(&st->ev[2], 1ull);
        if (u.u0 < Pb) {
          decay = true;
          bh = true;
          rmix = u.u1;   // the pair's energy split
        }
      }
    }
    if (live) {
      stv<R>(P.s1, i, xi.x); stv<R>(P.s2, i, xi.y); stv<R>(P.s3, i, xi.z);
      stv<R>(P.theta, i, th);
      P.x[i] = add_pos(x, dt * nn.x); P.y[i] = add_pos(y, dt * nn.y); P.z[i] = add_pos(z, dt * nn.z);
    }
    count_event(&st->ev[3], range);
    unsigned int r_in;
    const unsigned long long slot = tile_log(decay, tile, a.tile_cnt[0], &gst->cursor[0], a.rec_cap[0],
                                             &gst->status, s_tile, &r_in);
    if (slot != ~0ull) {
      NbwRec<R> rec;
      rec.i = i; rec.tile = tile; rec.r_in = r_in; rec.stamp = epoch;
      rec.ens = (unsigned int)ens | (bh ? kEvMedium : 0u);   // bit 31: a Bethe-Heitler decay
      rec.x = x; rec.y = y; rec.z = z;
      rec.chig = chig; rec.rmix = rmix; rec.p1x = P1.x; rec.p1y = P1.y; rec.p1z = P1.z;
      rec.kx = k.x; rec.ky = k.y; rec.kz = k.z; rec.x1 = xi.x; rec.x2 = xi.y; rec.x3 = xi.z;
      rec.w = ld<R>(P.w, i); rec.id = id;
      evlog[slot] = rec;
    }
    if constexpr (kPf) {
      cur = nxt;
      in = in_n;
    }
  }
}

// ---- Esirkepov current deposition (Sec. II C) with the TSC shape of Sec. II E, 2D3V ----
// The move (X0, Y0) -> (X1, Y1) in cell units (less than one cell per axis).  Shapes S0, S1
// on the 5 nodes around the old nearest node, DS = S1 - S0;
//   Wx = DS_x (S0_y + DS_y/2), Wy = DS_y (S0_x + DS_x/2),
//   Wz = S0_x S0_y + DS_x S0_y/2 + S0_x DS_y/2 + DS_x DS_y/3;
//   Jx(i+1/2,j) = -(q w/(dy dt)) sum_{i'<=i} Wx(i',j), Jy likewise along y,
//   Jz(i,j) = q w vz Wz(i,j)/(dx dy),
// so that (rho^{n+1} - rho^n)/dt + div J = 0 on the grid for the TSC charge of S0, S1.
// T is double on the FP64 path and float on the mixed one; J is float (the grid's type)
// and accumulated with atomic adds.
template <typename T>
__device__ __forceinline__ void tsc5(T X, int base, int shift, T S[5]) {
  // the 3 TSC weights of position X (nearest node base + shift) on nodes base-2..base+2
  const int ic = base + shift;
  const T d = X - T(ic);
#pragma unroll
  for (int k = 0; k < 5; ++k) S[k] = T(0);
  const T lo = T(0.5) - d, hi = T(0.5) + d;
  S[1 + shift] = T(0.5) * lo * lo;
  S[2 + shift] = T(0.75) - d * d;
  S[3 + shift] = T(0.5) * hi * hi;
}

// A lepton's move for the deposition, in cell units relative to the node (ib, jb), and its
// charge factors
template <typename T>
struct DepMove {
  T X0, Y0, X1, Y1;     // old and new position (cells, relative to node ib, jb)
  T cx, cy, cz;         // -q w/(dy dt), -q w/(dx dt), q w vz/(dx dy)
  int ib, jb;           // node the coordinates are relative to (FP64 path: 0)
  int i0, j0;           // old nearest node (absolute)
  bool on;              // live and within one cell per axis
};

template <typename T>
__device__ __forceinline__ void dep_move(DepMove<T>& m, T X0, T Y0, T X1, T Y1, T cx, T cy, T cz, int ib = 0,
                                         int jb = 0) {
  m.X0 = X0; m.Y0 = Y0; m.X1 = X1; m.Y1 = Y1; m.cx = cx; m.cy = cy; m.cz = cz;
  m.ib = ib; m.jb = jb;
  const int il = (int)floor(X0 + T(0.5)), jl = (int)floor(Y0 + T(0.5));
  m.i0 = ib + il;
  m.j0 = jb + jl;
  const int di = (int)floor(X1 + T(0.5)) - il, dj = (int)floor(Y1 + T(0.5)) - jl;
  m.on = di >= -1 && di <= 1 && dj >= -1 && dj <= 1;   // beyond the solver's CFL: not deposited
}

// Every term of the move on the support of its shapes goes to add(component, i, j, value),
// with the unwrapped node indices (i, j) of the component's position (Jx at i+1/2, Jy at
// j+1/2).  The support is the union of the old and new 3-node stencils: faces outside it
// carry no current (their cumulative sums vanish), so they are not visited.
template <typename T, typename Add>
__device__ __forceinline__ void esirkepov_terms(const DepMove<T>& m, Add add) {
  const int i0 = m.i0, j0 = m.j0;                 // absolute node indices of the adds
  const int il = i0 - m.ib, jl = j0 - m.jb;       // the same nodes in the move's local frame
  const int di = (int)floor(m.X1 + T(0.5)) - il, dj = (int)floor(m.Y1 + T(0.5)) - jl;
  T S0x[5], S1x[5], S0y[5], S1y[5];
  tsc5<T>(m.X0, il, 0, S0x);
  tsc5<T>(m.X1, il, di, S1x);
  tsc5<T>(m.Y0, jl, 0, S0y);
  tsc5<T>(m.Y1, jl, dj, S1y);
  const int cl = 1 + (di < 0 ? di : 0), ch = 3 + (di > 0 ? di : 0);
  const int bl = 1 + (dj < 0 ? dj : 0), bh = 3 + (dj > 0 ? dj : 0);
  // unrolled over the 5 stencil nodes (register arrays), predicated on the support
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if (b < bl || b > bh) continue;
    const T dsy = S1y[b] - S0y[b];
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      if (c < cl || c > ch) continue;
      const T dsx = S1x[c] - S0x[c];
      acc += dsx * (S0y[b] + T(0.5) * dsy);
      const T wz = S0x[c] * S0y[b] + T(0.5) * dsx * S0y[b] + T(0.5) * S0x[c] * dsy + dsx * dsy * T(1.0 / 3.0);
      if (c < ch && acc != T(0)) add(0, i0 - 2 + c, j0 - 2 + b, (float)(m.cx * acc));
      if (wz != T(0)) add(2, i0 - 2 + c, j0 - 2 + b, (float)(m.cz * wz));
    }
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (c < cl || c > ch) continue;
    const T dsx = S1x[c] - S0x[c];
    T acc = T(0);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (b < bl || b >= bh) continue;
      acc += (S1y[b] - S0y[b]) * (S0x[c] + T(0.5) * dsx);
      if (acc != T(0)) add(1, i0 - 2 + c, j0 - 2 + b, (float)(m.cy * acc));
    }
  }
}

// Deposition of one tile of leptons.  The current is first summed in a shared-memory
// window covering every stencil of the tile (tile-sorted particles share a few grid
// cells), then added to the grid once per window cell (float atomics); tiles whose stencils
// do not fit the window add every term to the grid directly.
// The window sums in fixed point: integer shared-memory atomics run at about three times
// the rate of float ones on this GPU, and integer sums do not depend on the order of the
// adds.  Each component has its own bound on a lepton's terms: a Jx term is cx times a
// cumulative sum of shape differences, whose magnitude is at most the move |X1 - X0| (its
// derivative in X is a linear B-spline, at most 1) times a weight of at most 1, so
// |term| <= |cx (X1 - X0)|; likewise |cy (Y1 - Y0)| for Jy, and |cz| for Jz (the averaged
// shape product is at most 1).  With b the tile's largest bound, b < 2^e, and the scale
// s = 2^(22 - e), a term is at most 2^22 units, and one cell collects at most 256 terms
// (one per lepton of the tile): below 2^30, inside int32.  Rounding a term to a multiple
// of 1/s < 2b 2^-22 costs about one float ulp of the tile's largest possible term.  For
// the lighter leptons of a tile whose weights spread widely that is coarse, so a tile whose
// largest charge factor exceeds 16 times its smallest sums the window in float instead.
// Window cells: with the staged rate tables the block's static shared memory stays below
// 48 KB (mixed: 16 KB of NCS interval cubics + 31 KB of window; FP64: 28 KB + 19 KB).
template <typename T> struct DepWin { static constexpr int v = sizeof(T) == 4 ? 2600 : 1600; };
template <typename T>
struct DepShared {
  int bnd[9];           // imin, imax, jmin, jmax of the tile's nearest nodes; largest term
                        // bound per component; largest and smallest positive |cx|
  int J[3 * DepWin<T>::v];   // int32 fixed point, or float (same bits for zero)
};
// the depositing lepton pass: window + staged tables + tile bookkeeping within 48 KB of
// static shared memory (1 KB left for the rest)
static_assert(sizeof(DepShared<float>) + sizeof(float) * kCoefLepLen + 1024 <= 48 * 1024, "mixed deposit smem");
static_assert(sizeof(DepShared<double>) + sizeof(double) * kSmemRateLen + 1024 <= 48 * 1024, "FP64 deposit smem");

template <typename T>
__device__ __forceinline__ void deposit_tile(const qed_fields& f, const DepMove<T>& m, DepShared<T>& sh) {
  const int nx = f.nx, ny = f.ny, per = f.periodic;
  float* const gJ[3] = {f.gJx, f.gJy, f.gJz};
  // per lepton: the bound of its terms of each component, and |cx| (its |q w| / (dy dt))
  const float bnd_m[4] = {(float)(fabs(m.cx) * fabs(m.X1 - m.X0)), (float)(fabs(m.cy) * fabs(m.Y1 - m.Y0)),
                          (float)fabs(m.cz), (float)fabs(m.cx)};
  block_bounds<4>(m.on, m.i0, m.j0, bnd_m, bnd_m[3], sh.bnd);
  const int imin = sh.bnd[0], imax = sh.bnd[1], jmin = sh.bnd[2], jmax = sh.bnd[3];
  if (imax < imin) {            // nothing to deposit in this tile
    __syncthreads();
    return;
  }
  const long long ww = (long long)imax - imin + 5, wh = (long long)jmax - jmin + 5;
  if (ww * wh <= DepWin<T>::v) {
    const int w = (int)ww, h = (int)wh, wi0 = imin - 2, wj0 = jmin - 2, nc = w * h;
    for (int k = threadIdx.x; k < 3 * nc; k += blockDim.x) sh.J[k] = 0;
    // fixed point unless the tile's charge factors spread by more than 16 (block-uniform)
    const bool fixed = __int_as_float(sh.bnd[7]) <= 16.0f * __int_as_float(sh.bnd[8]);
    float* const Jf = reinterpret_cast<float*>(sh.J);
    // per component the scale s = 2^(22 - e) with 2^e > its bound (frexpf: b = f 2^e, f < 1)
    float s[3], inv_s[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int e = 0;
      frexpf(__int_as_float(sh.bnd[4 + k]), &e);
      e = e < -100 ? -100 : e;
      s[k] = fixed ? ldexpf(1.0f, 22 - e) : 1.0f;
      inv_s[k] = fixed ? ldexpf(1.0f, e - 22) : 1.0f;
    }
    __syncthreads();
    if (m.on) {
      if (fixed) {
        DepMove<T> ms = m;
        ms.cx = m.cx * (T)s[0]; ms.cy = m.cy * (T)s[1]; ms.cz = m.cz * (T)s[2];
        esirkepov_terms<T>(ms, [&](int comp, int i, int j, float v) {
          atomicAdd(&sh.J[comp * nc + (j - wj0) * w + (i - wi0)], __float2int_rn(v));
        });
      } else {
        esirkepov_terms<T>(m, [&](int comp, int i, int j, float v) {
          atomicAdd(&Jf[comp * nc + (j - wj0) * w + (i - wi0)], v);
        });
      }
    }
    __syncthreads();
    // one warp per window row, lanes along the row
    const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int lj = threadIdx.x >> 5; lj < h; lj += nwarp) {
      const int gj = grid_node(wj0 + lj, ny, per);
      if (gj < 0) continue;
      for (int li = lane; li < w; li += 32) {
        const int gi = grid_node(wi0 + li, nx, per);
        if (gi < 0) continue;
        const size_t o = (size_t)gj * nx + gi;
        const int k = lj * w + li;
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
          const int v = sh.J[comp * nc + k];   // zero bits in both forms
          if (v != 0) atomicAdd(gJ[comp] + o, fixed ? (float)v * inv_s[comp] : __int_as_float(v));
        }
      }
    }
  } else if (m.on) {
    esirkepov_terms<T>(m, [&](int comp, int i, int j, float v) {
      const int gi = grid_node(i, nx, per), gj = grid_node(j, ny, per);
      if (gi >= 0 && gj >= 0) atomicAdd(gJ[comp] + (size_t)gj * nx + gi, v);
    });
  }
  __syncthreads();   // the window and its bounds are reused by the next tile
}

// ======================================================================================
// lepton streaming pass
// ======================================================================================
template <typename R, bool kB, bool kSm, bool kRad = false, bool kDep = false, bool kMed = false>
__global__ void __launch_bounds__(kTile, (kRad || kDep) ? OccPh<R>::v : Occ<R>::v)
    k_lepton(const __grid_constant__ StepArgs a) {
  __shared__ __align__(16) R s_rates[kSm ? SmemTab<R, false>::n : 1];
  __shared__ TileShared s_tile;
  __shared__ unsigned int s_off[kB ? kMaxEns + 1 : 1];
  __shared__ unsigned int s_et[kB ? kMaxEns : 1];
  __shared__ typename std::conditional<kDep, DepShared<R>, char>::type s_dep;
  DevState* gst = a.st;
  unsigned int ntiles, t0s = 0;
  unsigned long long n0s = 0, n1s = 0;   // single ensemble: its e-, e+ counts, read once
  if constexpr (kB) {
    for (int e = threadIdx.x; e <= a.n_ens; e += blockDim.x) {
      s_off[e] = a.map->lep_tile0[e];
      if (e < a.n_ens) s_et[e] = a.map->lep_e_tiles[e];
    }
    ntiles = a.map->lep_tile0[a.n_ens];
  } else {
    n0s = a.e0.sp[0].present ? a.e0.st->n_live[0] : 0ull;
    n1s = a.e0.sp[1].present ? a.e0.st->n_live[1] : 0ull;
    t0s = (unsigned int)((n0s + kTile - 1) / kTile);
    ntiles = t0s + (unsigned int)((n1s + kTile - 1) / kTile);
  }
  Tabs<R> tb = tabs_global<R>(a.tables);
  if constexpr (kSm) stage_rates<R, false>(tb, s_rates, &a.st->status);
  __syncthreads();
  const unsigned int epoch = gst->epoch;
  const R dt = sizeof(R) == 8 ? (R)a.dt : (R)a.fdt;
  NcsRec<R>* evlog = reinterpret_cast<NcsRec<R>*>(a.rec[1]);
  for (unsigned int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ens = kB ? find_ens_warp(s_off, a.n_ens, tile) : 0;
    const EnsArgs& E = ens_of<kB>(a, ens);
    const EnsTime tm = time_of<kB>(E);
    DevState* st = E.st;
    const unsigned int lt = tile - (kB ? s_off[ens] : 0u);     // tile inside the ensemble
    const unsigned int t0 = kB ? s_et[ens] : t0s;               // its e- tiles come first
    const int sp_idx = lt < t0 ? 0 : 1;
    const SpeciesArgs& L = E.sp[sp_idx];
    const unsigned long long nsp = kB ? (L.present ? st->n_live[sp_idx] : 0ull) : (sp_idx == 0 ? n0s : n1s);
    const unsigned int i = (lt - (sp_idx == 0 ? 0u : t0)) * kTile + threadIdx.x;
    const bool live = i < (unsigned int)nsp;
    const R q = sp_idx == 0 ? R(-1) : R(1);
    bool emit = false, range = false;
    DepMove<R> dm;
    dm.on = false;
    R chi = 0;
    V3<R> av = mk<R>(0, 0, 0);
    double x = 0.0, y = 0.0, z = 0.0;
    if (live) {
      x = L.x[i]; y = L.y[i]; z = L.z[i];
    }
    bool brems = false, in_med = false;
    if constexpr (kMed) in_med = live && in_medium(a, x, y, z);   // at x^n
    if (live) {
      V3<R> p = mk<R>(ld<R>(L.px, i), ld<R>(L.py, i), ld<R>(L.pz, i));
      V3<R> S = mk<R>(ld<R>(L.s1, i), ld<R>(L.s2, i), ld<R>(L.s3, i));
      const uint64_t id = L.id[i];
      const EB<R> f = gather<R, !kRad>(E, tm, x, y, z);
      // Boris push
      const R hq = R(0.5) * q * dt;
      const V3<R> pm = p + hq * f.E;
      const V3<R> tau = (hq * f_rsqrt(R(1) + dot(pm, pm))) * f.B;
      const V3<R> pp = pm + cross(pm, tau);
      const V3<R> sig = (R(2) * f_rcp(R(1) + dot(tau, tau))) * tau;
      V3<R> pn = pm + cross(pp, sig) + hq * f.E;
      RadSpin<R> rs;
      rs.on = false;
      if constexpr (kRad) {
        rad_push<R>(tb, a.flags, q, dt, f, p, pn, rs, range);
        if (rs.on) rad_spin_half<R>(rs, dt, S);
      }
      // T-BMT with beta, gamma of the mean of p^{n-1/2} and p^{n+1/2}
      if (a.flags & QED_F_SPIN) {
        const V3<R> pa = R(0.5) * (p + pn);
        const R ga2 = R(1) + dot(pa, pa);
        const R inv_ga = f_rsqrt(ga2);
        const R ga = ga2 * inv_ga;
        const V3<R> be = inv_ga * pa;
        const R inv_gp1 = f_rcp(ga + R(1));
        const R gg = ga * inv_gp1;
        const V3<R> Om = (-R(kAe) * gg * dot(be, f.B)) * be + (R(kAe) + inv_ga) * f.B +
                         (-(R(kAe) + inv_gp1)) * cross(be, f.E);
        const V3<R> tv = hq * Om;
        const V3<R> ov = (R(2) * f_rcp(R(1) + dot(tv, tv))) * tv;
        const V3<R> S1 = S + cross(S, tv);
        S = S + cross(S1, ov);
      }
      if constexpr (kRad) {
        if (rs.on) rad_spin_half<R>(rs, dt, S);
      }
      const R g12 = R(1) + dot(pn, pn);
      const R inv_g1 = f_rsqrt(g12);
      const R g1 = g12 * inv_g1;
      if (sizeof(R) == 8) {
        const double xo = x, yo = y;
        x += a.dt * (double)(pn.x / g1); y += a.dt * (double)(pn.y / g1); z += a.dt * (double)(pn.z / g1);
        if constexpr (kDep) {
          // the move x^n -> x^{n+1} in cell units, as the positions are stored
          const qed_fields& f = E.f;
          const double qw = (double)q * (double)ld<R>(L.w, i);
          dep_move<R>(dm, (xo - f.x0) / f.dx, (yo - f.y0) / f.dy, (x - f.x0) / f.dx, (y - f.y0) / f.dy,
                      -qw / (f.dy * a.dt), -qw / (f.dx * a.dt), qw * (double)(pn.z / g1) / (f.dx * f.dy));
        }
      } else {
        const R c = dt * inv_g1;
        if constexpr (kDep) {
          // cell coordinates as in the gather (node + float offset), the move from the float
          // displacement that the position update adds
          const Cell cx = cell_of(x, E.ff.gix, E.ff.gix_lo, E.ff.gox_i, E.ff.gox, E.ff.gox_lo);
          const Cell cy = cell_of(y, E.ff.giy, E.ff.giy_lo, E.ff.goy_i, E.ff.goy, E.ff.goy_lo);
          const float qw = (float)q * (float)ld<R>(L.w, i), idt = 1.0f / (float)dt;
          dep_move<R>(dm, cx.a, cy.a, cx.a + (float)(c * pn.x) * E.ff.gix, cy.a + (float)(c * pn.y) * E.ff.giy,
                      -qw * E.ff.giy * idt, -qw * E.ff.gix * idt, qw * (float)(c * pn.z) * idt * E.ff.gix * E.ff.giy,
                      cx.I, cy.I);
        }
        x = add_pos(x, c * pn.x); y = add_pos(y, c * pn.y); z = add_pos(z, c * pn.z);
      }
      if (a.flags & QED_F_NCS) {
        const R pm2 = dot(pn, pn);
        const R inv_pm = pm2 > R(0) ? f_rsqrt(pm2) : R(0);
        const V3<R> nn = inv_pm * pn;
        const R nE = dot(nn, f.E);
        V3<R> v = g1 * (f.E - nE * nn) + cross(pn, f.B);
        R vm2 = dot(v, v);
        if (sizeof(R) == 4) {
          // FP64 island: gamma E_perp and p x B cancel (co-propagation)
          const V3<R> a1 = g1 * (f.E - nE * nn), a2 = cross(pn, f.B);
          if (vm2 < R(1e-4) * (dot(a1, a1) + dot(a2, a2))) {
            const double px = pn.x, py = pn.y, pz = pn.z;
            const double G1 = sqrt(1.0 + px * px + py * py + pz * pz), pmd = sqrt(px * px + py * py + pz * pz);
            const double nx = px / pmd, ny = py / pmd, nz = pz / pmd;
            const double Ex = f.E.x, Ey = f.E.y, Ez = f.E.z, Bx = f.B.x, By = f.B.y, Bz = f.B.z;
            const double ne = nx * Ex + ny * Ey + nz * Ez;
            const double vx = G1 * (Ex - ne * nx) + (py * Bz - pz * By);
            const double vy = G1 * (Ey - ne * ny) + (pz * Bx - px * Bz);
            const double vz = G1 * (Ez - ne * nz) + (px * By - py * Bx);
            v = mk<R>((R)vx, (R)vy, (R)vz);
            vm2 = (R)(vx * vx + vy * vy + vz * vz);
          }
        }
        const R c2 = vm2 + nE * nE;
        chi = c2 > R(0) ? R(kXiL) * c2 * f_rsqrt(c2) : R(0);
        if (chi >= R(kChiMin) && vm2 > R(0) && inv_pm > R(0)) {
          if (chi > R(kChiMax)) { chi = R(kChiMax); range = true; }
          av = (q * f_rsqrt(vm2)) * v;    // unit acceleration direction
          const V3<R> zeta = cross(nn, av);
          R A, B;
          tb.ncs_rates(chi, A, B);
          const R s = dot(S, zeta);
          const R pref = R(kAlpha / (1.7320508075688772935 * kPi * kXiL)) * inv_g1;
          const R Wa = pref * A, Wb = pref * B;
          const R Pe = (Wa - s * Wb) * dt;
          const URand<R> u = urand<R, !kB>(E, id, tm.step, 0u);
          // one event per lepton per step is coarse where W dt > 0.1 (rare: no ballot)
          if (Pe > R(0.1)) atomicAdd(&st->ev[2], 1ull);
          if (u.u0 < Pe) {
            emit = true;   // completed by k_events
          } else {
            // no emission: posterior mean spin, then collapse with P(+) = (1+|S|)/2
            const R den = f_rcp(R(1) - Pe);
            const V3<R> Sb = (den * (R(1) - Wa * dt)) * S + (den * Wb * dt) * zeta;
            const R m2 = dot(Sb, Sb);
            const R inv_m = f_rsqrt(m2);
            const R sg = (u.u1 < R(0.5) * (R(1) + m2 * inv_m)) ? R(1) : R(-1);
            S = (sg * inv_m) * Sb;
          }
        }
      }
      if constexpr (kMed) {
        // bremsstrahlung in the medium, if no NCS event: P = 1 - exp(-n sigma(E) v dt) at the
        // energy of p^{n+1/2} (Sec. III E)
        const R pm2b = dot(pn, pn);
        if (!emit && in_med && (a.flags & QED_F_BREMS) && pm2b > R(0)) {
          const R sig = med_sigma<R>(a, 0, f_log(g1), range);
          const R Pb = -m_expm1(-R(a.med_nar2) * sig * (pm2b * f_rsqrt(pm2b)) * inv_g1 * dt);
          const URand<R> u = urand<R, !kB>(E, id, tm.step, 5u);
          if (Pb > R(0.1)) atomicAdd(&st->ev[2], 1ull);
          if (u.u0 < Pb) {
            emit = true;
            brems = true;
          }
        }
      }
      L.x[i] = x; L.y[i] = y; L.z[i] = z;
      stv<R>(L.px, i, pn.x); stv<R>(L.py, i, pn.y); stv<R>(L.pz, i, pn.z);
      stv<R>(L.s1, i, S.x); stv<R>(L.s2, i, S.y); stv<R>(L.s3, i, S.z);
    }
    if constexpr (kDep) deposit_tile<R>(E.f, dm, s_dep);
    count_event(&st->ev[sp_idx], emit && !brems);
    if constexpr (kMed) count_event(&st->ev[5 + sp_idx], brems);
    count_event(&st->ev[3], range);
    unsigned int r_in;
    const unsigned long long slot = tile_log(emit, tile, a.tile_cnt[1], &gst->cursor[1], a.rec_cap[1],
                                             &gst->status, s_tile, &r_in);
    if (slot != ~0ull) {
      NcsRec<R> rec;
      rec.i = i; rec.tile = tile; rec.r_in = r_in; rec.stamp = epoch;
      rec.species = (unsigned int)sp_idx | ((unsigned int)ens << 1) | (brems ? kEvMedium : 0u);   // bit 31: brems
      rec.chi = chi; rec.ax = av.x; rec.ay = av.y; rec.az = av.z;
      evlog[slot] = rec;
    }
  }
}

// ---- photon slots after a step ----------------------------------------------------------
// Decays leave holes h[0..D) (ascending).  With N photons at the step start and the new
// count M = N - D, the k-th surviving photon at or above M fills the k-th hole below M
// (both in index order), and the r-th birth takes slot M + r.  A birth into a slot below N
// first moves the photon there (if it survived) into its hole, and the slots at or above M
// that no birth takes are refill tasks of their own: so the refill, the births and the
// pair events (which read their photons from the log) run in one kernel in any order.
// Empty slot j (M <= j < N) of the photon set P: a surviving photon there moves to its hole.
// st carries D (n_nbw), M (n_surv) and the number of holes below M (n_hlow); h the holes.
template <typename R>
__device__ __noinline__ void ph_vacate(const SpeciesArgs& P, const DevState* st, const unsigned int* h,
                                       unsigned long long j) {
  // every load before the first store: the arrays may alias as far as the compiler knows,
  // and a load after a store would wait for the one before it
  const double x = P.x[j], y = P.y[j], z = P.z[j];
  const R px = ld<R>(P.px, j), py = ld<R>(P.py, j), pz = ld<R>(P.pz, j);
  const R s1 = ld<R>(P.s1, j), s2 = ld<R>(P.s2, j), s3 = ld<R>(P.s3, j);
  const R th = ld<R>(P.theta, j), w = ld<R>(P.w, j);
  const uint64_t id = P.id[j];
  const unsigned long long D = st->n_nbw, M = st->n_surv, H = st->n_hlow;
  unsigned long long lo = H, hi = D;   // the holes at or above M below j: h[H..lo)
  while (lo < hi) {
    const unsigned long long m = (lo + hi) >> 1;
    if ((unsigned long long)h[m] < j) lo = m + 1; else hi = m;
  }
  if (lo < D && (unsigned long long)h[lo] == j) return;   // slot j decayed
  const unsigned long long dst = h[(j - M) - (lo - H)];  // survivor rank among those at or above M
  P.x[dst] = x; P.y[dst] = y; P.z[dst] = z;
  stv<R>(P.px, dst, px); stv<R>(P.py, dst, py); stv<R>(P.pz, dst, pz);
  stv<R>(P.s1, dst, s1); stv<R>(P.s2, dst, s2); stv<R>(P.s3, dst, s3);
  stv<R>(P.theta, dst, th);
  stv<R>(P.w, dst, w);
  P.id[dst] = id;
}

// ======================================================================================
// exclusive scan of the tile counts (which = 0: photon tiles, 1: lepton tiles), one block;
// 32 consecutive counts per thread (vector loads) so that a pass covers 32768 tiles
// ======================================================================================
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 32;

// which < 0: both scans in one launch of two blocks (block 0 the photon tiles, block 1 the
// lepton tiles; they share nothing)
template <typename R, bool kB>
__global__ void __launch_bounds__(kScanThreads) k_scan(const __grid_constant__ StepArgs a, int which) {
  pdl_wait();
  pdl_trigger();
  if (which < 0) which = (int)blockIdx.x;
  __shared__ unsigned int s_w[kScanThreads / 32];
  __shared__ unsigned long long s_run;
  unsigned long long ntiles;
  if constexpr (kB) {
    ntiles = which == 0 ? a.map->ph_tile0[a.n_ens] : a.map->lep_tile0[a.n_ens];
  } else {
    const EnsArgs& E = a.e0;
    if (which == 0) {
      const unsigned long long nph = E.sp[2].present ? E.st->n_live[2] : 0ull;
      ntiles = (nph + kTile - 1) / kTile;
    } else {
      const unsigned long long n0 = E.sp[0].present ? E.st->n_live[0] : 0ull;
      const unsigned long long n1 = E.sp[1].present ? E.st->n_live[1] : 0ull;
      ntiles = (n0 + kTile - 1) / kTile + (n1 + kTile - 1) / kTile;
    }
  }
  const unsigned int* cnt = a.tile_cnt[which];
  unsigned int* pre = a.tile_pre[which];
  const unsigned int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  for (unsigned long long b = 0; b < ntiles; b += (unsigned long long)kScanThreads * kScanItems) {
    const unsigned long long first = b + (unsigned long long)threadIdx.x * kScanItems;
    const bool full = first + kScanItems <= ntiles;   // first is a multiple of 32: 16-byte aligned
    unsigned int v[kScanItems];
    if (full) {
      const uint4* c4 = reinterpret_cast<const uint4*>(cnt + first);
#pragma unroll
      for (int j = 0; j < kScanItems / 4; ++j) {
        const uint4 q = c4[j];
        v[4 * j] = q.x; v[4 * j + 1] = q.y; v[4 * j + 2] = q.z; v[4 * j + 3] = q.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < kScanItems; ++j) v[j] = (first + j < ntiles) ? cnt[first + j] : 0u;
    }
    unsigned int tsum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) tsum += v[j];
    unsigned int c = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, c, o);
      if (lane >= (unsigned)o) c += t;
    }
    if (lane == 31) s_w[warp] = c;
    __syncthreads();
    if (warp == 0) {
      unsigned int w = s_w[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= (unsigned)o) w += t;
      }
      s_w[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const unsigned long long run = s_run;
    unsigned int acc = (unsigned int)run + (warp ? s_w[warp - 1] : 0u) + c - tsum;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      const unsigned int e = acc;
      acc += v[j];
      v[j] = e;
    }
    if (full) {
      uint4* p4 = reinterpret_cast<uint4*>(pre + first);
#pragma unroll
      for (int j = 0; j < kScanItems / 4; ++j) p4[j] = make_uint4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < kScanItems; ++j)
        if (first + j < ntiles) pre[first + j] = v[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_run = run + s_w[kScanThreads / 32 - 1];
    __syncthreads();
  }
  // per-ensemble totals: an ensemble's events are the ranks between the prefixes at its
  // first tile and at the next ensemble's
  const int ne = kB ? a.n_ens : 1;
  const unsigned int* tile0 = kB ? (which == 0 ? a.map->ph_tile0 : a.map->lep_tile0) : nullptr;
  unsigned int* base = kB ? a.map->ev_base[which] : nullptr;
  if constexpr (kB) {
    __syncthreads();   // pre[] of this block is complete
    for (int e = threadIdx.x; e <= ne; e += blockDim.x)
      base[e] = tile0[e] < ntiles ? pre[tile0[e]] : (unsigned int)s_run;
    __syncthreads();
  }
  __shared__ unsigned long long s_m[kB ? kMaxEns : 1];    // new photon count M of each ensemble
  __shared__ unsigned int s_hl[kB ? kMaxEns : 1];         // its holes below M
  if (which == 0) {
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const EnsArgs& E = ens_of<kB>(a, e);
      const unsigned long long tot = kB ? (unsigned long long)(base[e + 1] - base[e]) : s_run;
      s_m[e] = (E.sp[2].present ? E.st->n_live[2] : 0ull) - tot;
      s_hl[e] = 0u;
    }
    __syncthreads();
    // the holes: the slot of every ranked decay at its rank (ascending slots per ensemble),
    // and how many lie below the ensemble's new count
    const DevState* gst = a.st;
    const unsigned long long nrec = min(gst->cursor[0], a.rec_cap[0]);
    const unsigned int epoch = gst->epoch;
    const NbwRec<R>* evlog = reinterpret_cast<const NbwRec<R>*>(a.rec[0]);
    for (unsigned long long kk = threadIdx.x; kk < nrec; kk += blockDim.x) {
      const NbwRec<R>& rec = evlog[kk];
      if (rec.stamp != epoch || cnt[rec.tile] == 0) continue;
      a.holes[pre[rec.tile] + rec.r_in] = (unsigned int)rec.i;
      const int ens = kB ? (int)(rec.ens & ~kEvMedium) : 0;
      if (rec.i < s_m[ens]) atomicAdd(&s_hl[ens], 1u);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const EnsArgs& E = ens_of<kB>(a, e);
    const unsigned long long tot = kB ? (unsigned long long)(base[e + 1] - base[e]) : s_run;
    if (which == 0) {
      E.st->n_nbw = tot;
      E.st->n_surv = s_m[e];
      E.st->n_hlow = s_hl[e];
    } else {
      E.st->n_ncs_tot = tot;
      if constexpr (!kB) {   // the e- tiles come first: their events are the first ranks
        const unsigned long long n0 = E.sp[0].present ? E.st->n_live[0] : 0ull;
        const unsigned long long te = (n0 + kTile - 1) / kTile;
        E.st->n_ncs_e = te < ntiles ? (unsigned long long)pre[te] : tot;
      }
    }
  }
}

// ======================================================================================
// NBW events: pair energy split (mixture over xi3' = +-1), SQAs D and D', joint spin
// sampling from Eqs. G0-G3, birth of the pair at the photon's x^n (Sec. III D)
// ======================================================================================
// A decay's pair as the decay leaves it: everything of its birth but the slots and ids.
template <typename R>
struct NbwPair {
  double x, y, z;    // the photon's x^n
  V3<R> p[2], s[2];  // momenta and spins, e- then e+
  R w;               // the photon's weight
};

// One decay (a task of k_events) up to its pair's slots.  It reads only its log entry and
// the tables, so it may run before the scan that ranks the events has finished.  Not inlined,
// so that the single-ensemble and the batched kernels run the same compiled arithmetic
// (inlined into different kernels, the compiler may fuse multiply-adds differently and
// results would differ in the last bit).  tcnt (the photon tile counts, or null): false
// when the entry's tile count is 0 (its log entries were dropped), loaded beside the work.
template <typename R>
__device__ __noinline__ bool nbw_pair(const NbwRec<R>& rec, const EnsArgs& E, const Tabs<R>& tb, unsigned int step,
                                      const unsigned int* tcnt, NbwPair<R>* out) {
  const bool tile_ok = tcnt == nullptr || tcnt[rec.tile] != 0u;
  const V3<R> k = mk<R>(rec.kx, rec.ky, rec.kz);
  const V3<R> xi = mk<R>(rec.x1, rec.x2, rec.x3);
  const R wgt = rec.w;
  const uint64_t id = rec.id;
  const R om = norm(k);
  const V3<R> nn = (R(1) / om) * k;
  const V3<R> P1 = mk<R>(rec.p1x, rec.p1y, rec.p1z);
  const V3<R> P2 = cross(nn, P1);
  const R chig = rec.chig;
  R T0, T3;
  tb.nbw_rates(chig, T0, T3);
  const Uni2 u2 = uniforms(E.seed, id, step, 4u);
  const R w0 = R(0.5) * (R(1) + xi.z) * (T0 - T3);
  const int comp = (rec.rmix * (T0 - xi.z * T3) < w0) ? 0 : 1;
  const double l = u2.u0;
  const bool upper = l >= 0.5;
  const double lam = upper ? 2.0 * (1.0 - l) : 2.0 * l;
  R tt = lam > 0.0 ? m_log((R)lam) : R(kBTLo);
  tt = tt < R(kBTLo) ? R(kBTLo) : tt;
  const R dh = m_exp(tb.nbw_inv(comp, chig, tt));
  R ep = upper ? (R(1) - dh) * om : dh * om;
  ep = ep < R(1) ? R(1) : ep;
  ep = ep > om - R(1) ? om - R(1) : ep;
  const R em = om - ep;
  const R delta = ep / om;
  R k13, k23, ik;
  tb.k(R(2) / (R(3) * chig * delta * (R(1) - delta)), k13, k23, ik);
  const R epm = ep * em;
  const R dif2 = (ep * ep - em * em) / epm, sum2 = (ep * ep + em * em) / epm, sq = (ep - em) * (ep - em) / epm;
  const R oe = om / ep, om_ = om / em;
  // SQAs: S+ along D (Eq. BWposAxis2), S- along D' (Eq. BWeleAxis1); a+ = P1', b+ = P2'
  const V3<R> D = (-(oe - xi.z * om_) * k13) * P2 + (-xi.x * om_ * k13) * P1 + (xi.y * (dif2 * k23 + oe * ik)) * nn;
  const V3<R> Dp = ((om_ - xi.z * oe) * k13) * P2 + (xi.x * oe * k13) * P1 + (-xi.y * (dif2 * k23 - om_ * ik)) * nn;
  const R dn = norm(D), dpn = norm(Dp);
  const V3<R> Sp = dn > R(0) ? (R(1) / dn) * D : P2;
  const V3<R> Sm = dpn > R(0) ? (R(1) / dpn) * Dp : P2;
  R pk[4];
  R tot = R(0);
  const R g2 = om * om / (R(2) * epm);
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const R sp = (o < 2) ? R(1) : R(-1), sm = (o % 2 == 0) ? R(1) : R(-1);
    const V3<R> A1 = sp * Sp, A2 = sm * Sm;
    const R SpSm = dot(A1, A2);
    const R Spb = dot(A1, P2), Smb = dot(A2, P2), Spa = dot(A1, P1), Sma = dot(A2, P1);
    const R Spv = dot(A1, nn), Smv = dot(A2, nn);
    const V3<R> X = cross(A2, A1);
    const R G0 = ik + sum2 * k23 + (ik - R(2) * k23) * SpSm + k13 * (-oe * Spb + om_ * Smb) +
                 (sum2 * ik - sq * k23) * Spv * Smv;
    const R G1 = k13 * (-om_ * Spa + oe * Sma) + R(0.5) * dif2 * k23 * dot(X, nn) - g2 * ik * (Spa * Smb + Sma * Spb);
    const R G2 = g2 * k13 * dot(X, P1) + R(0.5) * dif2 * k13 * (Smv * Spb + Spv * Smb) + (om_ * ik - dif2 * k23) * Smv +
                 (oe * ik + dif2 * k23) * Spv;
    const R G3 = -k23 + R(0.5) * sum2 * k23 * SpSm - k13 * (oe * Smb - om_ * Spb) + g2 * ik * (Spb * Smb - Spa * Sma) -
                 R(0.5) * sq * k23 * Spv * Smv;
    R v = G0 + xi.x * G1 + xi.y * G2 + xi.z * G3;
    v = v < R(0) ? R(0) : v;
    pk[o] = v;
    tot += v;
  }
  const R rr = (R)u2.u1 * tot;
  int o = 3;
  R acc = R(0);
#pragma unroll
  for (int qq = 0; qq < 4; ++qq) {
    acc += pk[qq];
    if (o == 3 && qq < 3 && rr < acc) o = qq;
  }
  const R sp = (o < 2) ? R(1) : R(-1), sm = (o % 2 == 0) ? R(1) : R(-1);
  const R pp = sqrt(ep * ep - R(1)), pm = sqrt(em * em - R(1));
  if (!tile_ok) return false;
  out->x = rec.x; out->y = rec.y; out->z = rec.z;
  out->p[0] = mk<R>(pm * nn.x, pm * nn.y, pm * nn.z);
  out->p[1] = mk<R>(pp * nn.x, pp * nn.y, pp * nn.z);
  out->s[0] = sm * Sm;
  out->s[1] = sp * Sp;
  out->w = wgt;
  return true;
}

// The pair of the decay of rank `rank` takes slot n_live + rank of each lepton set, with
// ids next_id + 2 rank (e-) and + 1 (e+).  Needs the scan's rank only.
template <typename R>
__device__ __forceinline__ void nbw_birth(const NbwPair<R>& q, const EnsArgs& E, unsigned long long rank,
                                          DevState* gst) {
  DevState* st = E.st;
  const unsigned long long base[2] = {st->n_live[0], st->n_live[1]};
  const unsigned long long id0 = st->next_id + st->id_add[0];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const SpeciesArgs& L = E.sp[s];
    const unsigned long long j = base[s] + rank;
    if (!L.present || j >= L.cap) {
      atomicOr(&gst->status, QED_STATUS_CAPACITY);
      atomicAdd(&st->ev[4], 1ull);
      continue;
    }
    L.x[j] = q.x; L.y[j] = q.y; L.z[j] = q.z;
    stv<R>(L.px, j, q.p[s].x); stv<R>(L.py, j, q.p[s].y); stv<R>(L.pz, j, q.p[s].z);
    stv<R>(L.s1, j, q.s[s].x); stv<R>(L.s2, j, q.s[s].y); stv<R>(L.s3, j, q.s[s].z);
    stv<R>(L.w, j, q.w);
    L.id[j] = id0 + 2ull * rank + (unsigned long long)s;
  }
}

// a whole decay, once the scan has finished
template <typename R>
__device__ __forceinline__ void nbw_event(const NbwRec<R>& rec, const EnsArgs& E, const Tabs<R>& tb, unsigned int step,
                                          unsigned long long rank, DevState* gst) {
  NbwPair<R> q;
  nbw_pair<R>(rec, E, tb, step, nullptr, &q);
  nbw_birth<R>(q, E, rank, gst);
}

// ---- matter events (Sec. III E) ------------------------------------------------------
// A Bethe-Heitler decay: the positron takes x k (x from the cumulative cross-section with
// the uniform carried in rec.rmix), the electron k - x k (each at least m c^2), both along
// the photon, born at its x^n with S = 0 (unpolarised) and the photon's weight.
template <typename R>
__device__ __noinline__ void bh_event(const StepArgs& a, const NbwRec<R>& rec, const EnsArgs& E, unsigned long long rank,
                                      DevState* gst) {
  DevState* st = E.st;
  const unsigned long long ne0 = st->n_live[0], np0 = st->n_live[1], id0 = st->next_id + st->id_add[0];
  const double kx = (double)rec.kx, ky = (double)rec.ky, kz = (double)rec.kz;
  const R wgt = rec.w;
  const double om = sqrt(kx * kx + ky * ky + kz * kz);
  const double nx = kx / om, ny = ky / om, nz = kz / om;
  const double xf = med_sample(a, 1, om, (double)rec.rmix);
  double ep = xf * om;
  ep = ep < 1.0 ? 1.0 : ep;
  ep = ep > om - 1.0 ? om - 1.0 : ep;
  const double em = om - ep;
  const double pmag[2] = {sqrt(em * em - 1.0), sqrt(ep * ep - 1.0)};   // e-, e+
  const unsigned long long base[2] = {ne0, np0};
  atomicAdd(&st->ev[7], 1ull);
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const SpeciesArgs& L = E.sp[sp];
    const unsigned long long j = base[sp] + rank;
    if (!L.present || j >= L.cap) {
      atomicOr(&gst->status, QED_STATUS_CAPACITY);
      atomicAdd(&st->ev[4], 1ull);
      continue;
    }
    L.x[j] = rec.x; L.y[j] = rec.y; L.z[j] = rec.z;
    stv<R>(L.px, j, (R)(pmag[sp] * nx)); stv<R>(L.py, j, (R)(pmag[sp] * ny)); stv<R>(L.pz, j, (R)(pmag[sp] * nz));
    stv<R>(L.s1, j, R(0)); stv<R>(L.s2, j, R(0)); stv<R>(L.s3, j, R(0));
    stv<R>(L.w, j, wgt);
    L.id[j] = id0 + 2ull * rank + (unsigned long long)sp;
  }
}

// A bremsstrahlung emission: omega = y E (y from the cumulative cross-section with the
// second uniform of the decision's draw), along p; the lepton keeps its direction with
// energy E - omega and its spin; the photon is unpolarised (xi = 0, basis angle 0), born
// at the lepton's x^{n+1}.
template <typename R>
__device__ __noinline__ void brems_event(const StepArgs& a, const NcsRec<R>& rec, const EnsArgs& E, unsigned int step,
                                         unsigned long long rank, bool births, unsigned int flags, DevState* gst,
                                         const unsigned int* holes) {
  DevState* st = E.st;
  const SpeciesArgs& G = E.sp[2];
  const SpeciesArgs& L = E.sp[rec.species & 1u];
  const unsigned long long nsurv = st->n_surv;
  const unsigned long long id0 = st->next_id + 2ull * st->n_nbw + st->id_add[1u + (rec.species & 1u)];
  const unsigned long long nph0 = st->n_live[2];
  const unsigned long long i = rec.i;
  const double px = (double)ld<R>(L.px, i), py = (double)ld<R>(L.py, i), pz = (double)ld<R>(L.pz, i);
  const double lx = L.x[i], ly = L.y[i], lz = L.z[i];   // read before the lepton's stores
  const R lw = ld<R>(L.w, i);
  const double pmag = sqrt(px * px + py * py + pz * pz);
  if (!(pmag > 0.0)) return;
  const double g1 = sqrt(1.0 + px * px + py * py + pz * pz);
  const Uni2 u = uniforms(E.seed, L.id[i], step, 5u);
  const double yv = med_sample(a, 0, g1, u.u1);
  const double om = yv * g1;
  double gf = g1 - om;
  gf = gf < 1.0 ? 1.0 : gf;
  const double nx = px / pmag, ny = py / pmag, nz = pz / pmag;
  if (!(flags & QED_F_NO_RECOIL)) {
    const double pf = sqrt(gf * gf - 1.0);
    stv<R>(L.px, i, (R)(pf * nx)); stv<R>(L.py, i, (R)(pf * ny)); stv<R>(L.pz, i, (R)(pf * nz));
  }
  if (births) {
    const unsigned long long j = nsurv + rank;
    if (!G.present || j >= G.cap) {
      atomicOr(&gst->status, QED_STATUS_CAPACITY);
      atomicAdd(&st->ev[4], 1ull);
    } else {
      if (j < nph0) ph_vacate<R>(G, st, holes, j);
      G.x[j] = lx; G.y[j] = ly; G.z[j] = lz;
      stv<R>(G.px, j, (R)(om * nx)); stv<R>(G.py, j, (R)(om * ny)); stv<R>(G.pz, j, (R)(om * nz));
      stv<R>(G.s1, j, R(0)); stv<R>(G.s2, j, R(0)); stv<R>(G.s3, j, R(0));
      stv<R>(G.theta, j, R(0));
      stv<R>(G.w, j, lw);
      G.id[j] = id0 + rank;
    }
  }
}

// ======================================================================================
// NCS events: photon energy (two-component mixture of Eq. Wspin2 at s = S.zeta), recoil,
// spin collapse along the SQA of Eq. F0, photon pure state from Eqs. F1-F3, photon birth
// at x^{n+1}; the last block to finish closes the step.
// ======================================================================================
// The last block of the final event kernel closes the step: counts, id counters,
// statistics, clocks (batched), resets.  Called by every block of that kernel.
template <bool kB>
__device__ __forceinline__ void close_step(const StepArgs& a, bool births) {
  DevState* gst = a.st;
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int d = atomicAdd(&gst->done, 1u);
    s_last = d == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const unsigned int epoch = threadIdx.x == 0 ? static_cast<volatile DevState*>(gst)->epoch : 0u;
  const int ne = kB ? a.n_ens : 1;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const EnsArgs& E = ens_of<kB>(a, e);
    volatile DevState* v = E.st;
    // every load before the first store: one round trip
    const unsigned long long nbw = v->n_nbw, ncs = births ? v->n_ncs_tot : 0ull, surv = v->n_surv;
    const unsigned long long live[3] = {v->n_live[0], v->n_live[1], v->n_live[2]};
    const unsigned long long nid = v->next_id, add3 = v->id_add[3];
    unsigned long long ev[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ev[q] = v->ev[q];
    const double t0 = kB ? v->t : 0.0;
    const unsigned int step0 = kB ? v->step : 0u;
    const unsigned long long processed = (E.sp[0].present ? live[0] : 0ull) +   // step-start counts
                                         (E.sp[1].present ? live[1] : 0ull) +
                                         (E.sp[2].present ? live[2] : 0ull);
    for (int s = 0; s < 2; ++s) {
      if (!E.sp[s].present) continue;
      const unsigned long long nn = live[s] + nbw;
      v->n_live[s] = nn > E.sp[s].cap ? E.sp[s].cap : nn;
    }
    if (E.sp[2].present) {
      const unsigned long long nn = surv + ncs;
      v->n_live[2] = nn > E.sp[2].cap ? E.sp[2].cap : nn;
    }
    v->next_id = nid + 2ull * nbw + ncs + add3;
    atomicAdd(&gst->processed, processed);
    if (E.user_stats) {
      E.user_stats->n_processed += processed;
      E.user_stats->n_ncs[0] += ev[0];
      E.user_stats->n_ncs[1] += ev[1];
      E.user_stats->n_nbw += nbw - ev[7];   // the ranked decays include the Bethe-Heitler pairs
      E.user_stats->n_brems[0] += ev[5];
      E.user_stats->n_brems[1] += ev[6];
      E.user_stats->n_bh += ev[7];
      E.user_stats->n_range += ev[3];
      E.user_stats->n_drop += ev[4];
      E.user_stats->n_steps += 1;
      E.user_stats->n_coarse += ev[2];
    }
    if (ev[3]) atomicOr(&gst->status, QED_STATUS_TABLE_RANGE);
    for (int q = 0; q < 8; ++q) v->ev[q] = 0;
    v->n_nbw = 0; v->n_surv = 0; v->n_ncs_tot = 0; v->n_hlow = 0; v->n_ncs_e = 0;
    for (int q = 0; q < 4; ++q) v->id_add[q] = 0;
    if constexpr (kB) {
      // the ensemble's clock: the same operations as the host forms of a single step
      const double t = t0 + a.dt;
      v->t = t;
      v->step = step0 + 1;
      v->t_rel = (float)(t - E.f.phi0);
      v->t_mod = (float)fma(-kTwoPi, floor(t / kTwoPi), t);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // the kernel's end publishes these to the next step's kernels
    volatile DevState* g = gst;
    g->cursor[0] = 0; g->cursor[1] = 0;
    g->done = 0;
    g->epoch = epoch + 1;
  }
}

// An emitted photon as its emission leaves it: everything of its birth but the slot and id.
template <typename R>
struct NcsBirth {
  double x, y, z;   // the lepton's x^{n+1}
  V3<R> k, xi;      // omega n and the pure Stokes state
  R theta, w;       // basis angle of the Stokes frame, weight
};

// One emission (a task of k_events) up to its photon's slot: energy, recoil, spin collapse
// and the photon's state (written to *out when births are on).  It reads only the lepton,
// its log entry and the tables, and writes only the lepton, so it may run before the scan
// that ranks the events has finished.  Not inlined for the same reason as nbw_pair.
// tcnt (the lepton tile counts, or null): when the entry's tile count is 0 (its log entries
// were dropped) the emission writes nothing and returns false; the count is loaded with
// the lepton instead of before it.
template <typename R>
__device__ __noinline__ bool ncs_emit(const NcsRec<R>& rec, const EnsArgs& E, const Tabs<R>& tb, unsigned int step,
                                      bool births, unsigned int flags, bool learned, float lnu_learned,
                                      const unsigned int* tcnt, NcsBirth<R>* out) {
  const bool tile_ok = tcnt == nullptr || tcnt[rec.tile] != 0u;
  const SpeciesArgs& L = E.sp[rec.species & 1u];
  const unsigned long long i = rec.i;
  const V3<R> pn = mk<R>(ld<R>(L.px, i), ld<R>(L.py, i), ld<R>(L.pz, i));
  const V3<R> S = mk<R>(ld<R>(L.s1, i), ld<R>(L.s2, i), ld<R>(L.s3, i));
  const uint64_t id = L.id[i];
  const double lx = L.x[i], ly = L.y[i], lz = L.z[i];   // the photon's birth place and weight,
  const R lw = ld<R>(L.w, i);                            // read before the lepton's stores
  const R chi = rec.chi;
  const V3<R> av = mk<R>(rec.ax, rec.ay, rec.az);
  const R g1 = sqrt(R(1) + dot(pn, pn));
  R pmag = norm(pn);
  pmag = pmag > R(0) ? pmag : R(1e-30);
  const V3<R> nn = (R(1) / pmag) * pn;
  const V3<R> zeta = cross(nn, av);
  R A, B;
  tb.ncs_rates(chi, A, B);
  const R s = dot(S, zeta);
  const Uni2 um = uniforms(E.seed, id, step, 1u);
  const Uni2 us = uniforms(E.seed, id, step, 2u);
  R uu;
  if (learned) {
    uu = (R)expf(lnu_learned);   // the learned sampler's ln u (one uniform, um.u1)
  } else {
    const R wplus = R(0.5) * (R(1) + s) * (A - B);
    const int comp = ((R)um.u0 * (A - s * B) < wplus) ? 0 : 1;
    const double l = um.u1;
    R tt;
    if (sizeof(R) == 8) tt = (R)(log(l) - log1p(-l));
    else tt = m_log((R)l) - m_log((R)(1.0 - l));
    tt = tt < R(kCTLo) ? R(kCTLo) : (tt > R(kCTHi) ? R(kCTHi) : tt);
    uu = m_exp(tb.ncs_inv(comp, chi, tt));
  }
  const R omr = R(1) / (R(1) + uu), rr = uu * omr;
  const R om = rr * g1;
  R k13, k23, ik;
  tb.k(R(2) * uu / (R(3) * chi), k13, k23, ik);
  const R sin_ = dot(S, nn);
  const R c0 = R(4) * ((R(2) + R(2) * uu + uu * uu) * k23 - (R(1) + uu) * ik - uu * s * k13);
  const V3<R> gv = (R(-4) * (R(1) + uu) * (ik - R(2) * k23)) * S + (R(-4) * uu * (R(1) + uu) * k13) * zeta +
                   (R(-4) * uu * uu * (ik - k23) * sin_) * nn;
  const R gmg = norm(gv);
  V3<R> Sf = S;
  if (gmg > R(0)) {
    const R sg = ((R)us.u0 < R(0.5) * (R(1) + gmg / c0)) ? R(1) : R(-1);
    Sf = (sg / gmg) * gv;
  }
  const R F0 = c0 + dot(gv, Sf);
  const R Sif = dot(S, Sf), Siz = s, Sfz = dot(Sf, zeta), Sin = sin_, Sfn = dot(Sf, nn);
  const R Sia = dot(S, av), Sfa = dot(Sf, av);
  const V3<R> fxs = cross(Sf, S);
  const R u2 = uu * uu;
  const R F1 = R(-2) * u2 * ik * (Sia * Sfz + Sfa * Siz) + R(4) * uu * (Sia * (R(1) + uu) + Sfa) * k13 +
               R(2) * uu * (R(2) + uu) * dot(nn, fxs) * k23;
  const R F2 = -(R(2) * u2 * (Sin * Sfz + Sfn * Siz) + R(2) * uu * (R(2) + uu) * dot(av, fxs)) * k13 -
               R(4) * uu * (Sin + Sfn * (R(1) + uu)) * ik + R(4) * uu * (R(2) + uu) * (Sin + Sfn) * k23;
  const R F3 = R(4) * (R(1) + uu + (R(1) + uu + R(0.5) * u2) * Sif - R(0.5) * u2 * Sin * Sfn) * k23 +
               R(2) * u2 * (Siz * Sfz - Sia * Sfa) * ik - R(4) * uu * ((R(1) + uu) * Siz + Sfz) * k13;
  const R fm = sqrt(F1 * F1 + F2 * F2 + F3 * F3);
  V3<R> xiph = mk<R>(0, 0, 0);
  if (fm > R(0)) {
    const R sg = ((R)us.u1 < R(0.5) * (R(1) + fm / F0)) ? R(1) : R(-1);
    xiph = mk<R>(sg * F1 / fm, sg * F2 / fm, sg * F3 / fm);
  }
  if (!tile_ok) return false;
  stv<R>(L.s1, i, Sf.x); stv<R>(L.s2, i, Sf.y); stv<R>(L.s3, i, Sf.z);
  if (!(flags & QED_F_NO_RECOIL)) {
    // recoil p_f = p_i - omega n, |p_f| = (1-r) gamma - (gamma - |p|)
    const R pf = omr * g1 - R(1) / (g1 + pmag);
    stv<R>(L.px, i, pf * nn.x); stv<R>(L.py, i, pf * nn.y); stv<R>(L.pz, i, pf * nn.z);
  }
  if (births) {
    V3<R> e1, e2;
    frame(nn, e1, e2);
    out->x = lx; out->y = ly; out->z = lz;
    out->k = mk<R>(om * nn.x, om * nn.y, om * nn.z);
    out->xi = xiph;
    out->theta = m_atan2(dot(av, e2), dot(av, e1));
    out->w = lw;
  }
  return true;
}

// The photon of the emission of rank `rank` (species: its lepton's log tag) takes slot
// n_surv + rank, after the survivor there has moved to its hole; its id is the next free one
// after the step's pairs.  Needs the scan's counts and holes.
template <typename R>
__device__ __forceinline__ void ncs_birth(const NcsBirth<R>& b, const EnsArgs& E, unsigned int species,
                                          unsigned long long rank, DevState* gst, const unsigned int* holes) {
  DevState* st = E.st;
  const SpeciesArgs& G = E.sp[2];
  const unsigned long long nsurv = st->n_surv, nph0 = st->n_live[2];
  const unsigned long long id0 = st->next_id + 2ull * st->n_nbw + st->id_add[1u + (species & 1u)];
  const unsigned long long j = nsurv + rank;
  if (!G.present || j >= G.cap) {
    atomicOr(&gst->status, QED_STATUS_CAPACITY);
    atomicAdd(&st->ev[4], 1ull);
    return;
  }
  if (j < nph0) ph_vacate<R>(G, st, holes, j);
  G.x[j] = b.x; G.y[j] = b.y; G.z[j] = b.z;
  stv<R>(G.px, j, b.k.x); stv<R>(G.py, j, b.k.y); stv<R>(G.pz, j, b.k.z);
  stv<R>(G.s1, j, b.xi.x); stv<R>(G.s2, j, b.xi.y); stv<R>(G.s3, j, b.xi.z);
  stv<R>(G.theta, j, b.theta);
  stv<R>(G.w, j, b.w);
  G.id[j] = id0 + rank;
}

// a whole emission, once the scan has finished
template <typename R>
__device__ __forceinline__ void ncs_event(const NcsRec<R>& rec, const EnsArgs& E, const Tabs<R>& tb, unsigned int step,
                                          unsigned long long rank, bool births, unsigned int flags, DevState* gst,
                                          bool learned, float lnu_learned, const unsigned int* holes) {
  NcsBirth<R> b;
  ncs_emit<R>(rec, E, tb, step, births, flags, learned, lnu_learned, nullptr, &b);
  if (births) ncs_birth<R>(b, E, rec.species, rank, gst, holes);
}

// ---- sharded steps: one rank's birth counts; the id offsets from every rank's -------------
// counts = (pairs, e- emissions, e+ emissions); without births (QED_F_NO_RECOIL,
// QED_F_DROP_PHOTONS) the emissions take no ids and count zero
static __global__ void k_shard_counts(const __grid_constant__ StepArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const DevState* st = a.e0.st;
  const bool births = !(a.flags & (QED_F_NO_RECOIL | QED_F_DROP_PHOTONS));
  a.shard_counts[0] = st->n_nbw;
  a.shard_counts[1] = births ? st->n_ncs_e : 0ull;
  a.shard_counts[2] = births ? st->n_ncs_tot - st->n_ncs_e : 0ull;
}

// The step's births on all ranks numbered as one sequential pass over the ranks' particles
// in rank order would number them: all pairs, then every e- emission, then every e+
// emission.  With P, E, Q the counts of the ranks before this one and TP, TE, TQ the totals,
// a pair k gets next + 2 (P + k) + s, an e- emission k next + 2 TP + E + k, an e+ emission k
// next + 2 TP + TE + Q + k, and the counter moves to next + 2 TP + TE + TQ: the offsets
// against this rank's own numbering go to id_add.  A rank whose gathered counts are not its
// own sets QED_STATUS_SHARD (the ids would collide).
static __global__ void k_shard_ids(const __grid_constant__ StepArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DevState* st = a.e0.st;
  const bool births = !(a.flags & (QED_F_NO_RECOIL | QED_F_DROP_PHOTONS));
  const unsigned long long own[3] = {st->n_nbw, births ? st->n_ncs_e : 0ull,
                                     births ? st->n_ncs_tot - st->n_ncs_e : 0ull};
  unsigned long long before[3] = {0ull, 0ull, 0ull}, tot[3] = {0ull, 0ull, 0ull};
  for (int q = 0; q < a.shard_world; ++q)
    for (int k = 0; k < 3; ++k) {
      const unsigned long long v = a.shard_all[3 * q + k];
      tot[k] += v;
      if (q < a.shard_rank) before[k] += v;
    }
  for (int k = 0; k < 3; ++k)
    if (a.shard_all[3 * a.shard_rank + k] != own[k]) atomicOr(&a.st->status, QED_STATUS_SHARD);
  const unsigned long long dp = 2ull * (tot[0] - own[0]);   // unsigned: offsets wrap mod 2^64
  st->id_add[0] = 2ull * before[0];
  st->id_add[1] = dp + before[1];
  st->id_add[2] = dp + tot[1] + before[2] - own[1];
  st->id_add[3] = dp + (tot[1] + tot[2]) - (own[1] + own[2]);
}

// ---- the event kernel's tasks ----------------------------------------------------------
// The ensemble's holes (its ranked decays' slots, ascending)
template <bool kB>
__device__ __forceinline__ const unsigned int* holes_of(const StepArgs& a, int ens) {
  return a.holes + (kB ? a.map->ev_base[0][ens] : 0u);
}

// one logged decay: NBW (Sec. III D) or Bethe-Heitler (Sec. III E) pair creation
template <typename R, bool kB>
__device__ __forceinline__ void nbw_task(const StepArgs& a, const Tabs<R>& tb, const NbwRec<R>& rec,
                                         unsigned int epoch, DevState* gst) {
  if (rec.stamp != epoch || a.tile_cnt[0][rec.tile] == 0) return;
  const unsigned int ens = rec.ens & ~kEvMedium;
  const EnsArgs& E = ens_of<kB>(a, kB ? (int)ens : 0);
  // global rank (index of the ranked hole) and rank inside the ensemble
  const unsigned long long grank = (unsigned long long)a.tile_pre[0][rec.tile] + rec.r_in;
  const unsigned long long rank = kB ? grank - a.map->ev_base[0][ens] : grank;
  if (rec.ens & kEvMedium) bh_event<R>(a, rec, E, rank, gst);
  else nbw_event<R>(rec, E, tb, time_of<kB>(E).step, rank, gst);
}

// refill task f: slot M + r of its ensemble, for the r (C <= r < D) that no birth takes
template <typename R, bool kB>
__device__ __forceinline__ void fill_task(const StepArgs& a, const unsigned int* s_fb, unsigned long long f) {
  const int ens = kB ? find_ens(s_fb, a.n_ens, (unsigned int)f) : 0;
  const EnsArgs& E = ens_of<kB>(a, ens);
  const DevState* st = E.st;
  const unsigned long long D = st->n_nbw;
  const unsigned long long nf = kB ? (unsigned long long)(s_fb[ens + 1] - s_fb[ens]) : s_fb[0];
  const unsigned long long r = (D - nf) + (f - (kB ? s_fb[ens] : 0u));
  ph_vacate<R>(E.sp[2], st, holes_of<kB>(a, ens), st->n_surv + r);
}

// the number of refill tasks (single ensemble) or their per-ensemble bases (batched: the
// refill tasks of ensemble e are its slots M + r, C <= r < D, that no birth takes)
template <bool kB>
__device__ __forceinline__ unsigned long long fill_setup(const StepArgs& a, bool births, unsigned int* s_fb) {
  if constexpr (kB) {
    // every ensemble's count by its own thread (the loads in parallel), then the prefix in
    // shared memory
    for (int e = threadIdx.x; e < a.n_ens; e += blockDim.x) {
      const DevState* st = ens_of<kB>(a, e).st;
      const unsigned long long D = st->n_nbw, C = births ? st->n_ncs_tot : 0ull;
      s_fb[e + 1] = (unsigned int)(C < D ? D - C : 0ull);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int f = 0;
      s_fb[0] = 0u;
      for (int e = 1; e <= a.n_ens; ++e) {
        f += s_fb[e];
        s_fb[e] = f;
      }
    }
    __syncthreads();
    return s_fb[a.n_ens];
  } else {
    const DevState* st = a.e0.st;
    const unsigned long long D = st->n_nbw, C = births ? st->n_ncs_tot : 0ull;
    s_fb[0] = (unsigned int)(C < D ? D - C : 0ull);
    return C < D ? D - C : 0ull;
  }
}

// ======================================================================================
// k_events: every logged emission, every logged decay and every refill task of the step,
// one thread each (grid-stride); they touch disjoint data (see the photon-slot rules
// above), so one launch runs them all.  Its last block closes the step.
//
// It is launched as a programmatic dependent of the scan, which is an ordinary launch after
// both streaming passes: when it starts, the passes have finished and only the scan's
// results (ranks, holes, counts) may still be missing.  So each thread takes its first
// emission or decay up to the rank-dependent birth before it waits for the scan, and the
// sampling and spin arithmetic of the step's events runs beside the scan.
// ======================================================================================
template <typename R, bool kB>
// Batched launches carry ~1e5 events a step and are throughput-bound: four blocks per SM
// (64 registers, some spills) step the 64-ensemble batch 1% faster than two; a single
// ensemble's few thousand events are latency-bound and keep the registers (0: no minimum).
__global__ void __launch_bounds__(kTile, kB ? 4 : 0) k_events(const __grid_constant__ StepArgs a) {
  __shared__ unsigned int s_fb[kB ? kMaxEns + 1 : 1];
  DevState* gst = a.st;
  const Tabs<R> tb = tabs_global<R>(a.tables);
  // the logs, their extents and the tile counts are the passes' (final here)
  const unsigned long long n1 = min(gst->cursor[1], a.rec_cap[1]);
  const unsigned long long n0 = min(gst->cursor[0], a.rec_cap[0]);
  const unsigned int epoch = gst->epoch;
  const bool births = !(a.flags & (QED_F_NO_RECOIL | QED_F_DROP_PHOTONS));
  const NcsRec<R>* ncslog = reinterpret_cast<const NcsRec<R>*>(a.rec[1]);
  const NbwRec<R>* nbwlog = reinterpret_cast<const NbwRec<R>*>(a.rec[0]);
  const unsigned long long k0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  // the first task, before the scan: 1 an emission, 2 a decay (NBW), taken up to the birth
  int early = 0;
  unsigned int e_tile = 0u, e_rin = 0u, e_tag = 0u;
  NcsBirth<R> eb;
  NbwPair<R> ep;
  if (k0 < a.rec_cap[1]) {
    // the emission record is read beside the log extents (a stale entry fails the stamp)
    const NcsRec<R> rec = ncslog[k0];
    if (k0 < n1 && rec.stamp == epoch && !(rec.species & kEvMedium)) {
      const EnsArgs& E = ens_of<kB>(a, kB ? (int)(rec.species >> 1) : 0);
      if (ncs_emit<R>(rec, E, tb, time_of<kB>(E).step, births, a.flags, false, 0.0f, a.tile_cnt[1], &eb)) {
        early = 1; e_tile = rec.tile; e_rin = rec.r_in; e_tag = rec.species;
      }
    }
  }
  if (k0 >= n1 && k0 < n1 + n0) {
    const NbwRec<R> rec = nbwlog[k0 - n1];
    if (rec.stamp == epoch && !(rec.ens & kEvMedium)) {
      const EnsArgs& E = ens_of<kB>(a, kB ? (int)rec.ens : 0);
      if (nbw_pair<R>(rec, E, tb, time_of<kB>(E).step, a.tile_cnt[0], &ep)) {
        early = 2; e_tile = rec.tile; e_rin = rec.r_in; e_tag = rec.ens;
      }
    }
  }
  pdl_wait();
  // the first task's birth: its rank and the counts it needs in one round trip (the refill
  // set-up, which stores to shared memory, comes after it)
  if (early != 0) {
    const int e_ens = kB ? (int)(early == 1 ? e_tag >> 1 : e_tag) : 0;
    const int w = early == 1 ? 1 : 0;
    unsigned long long e_rank = (unsigned long long)a.tile_pre[w][e_tile] + e_rin;
    if constexpr (kB) e_rank -= a.map->ev_base[w][e_ens];
    if (early == 1) {
      if (births) ncs_birth<R>(eb, ens_of<kB>(a, e_ens), e_tag, e_rank, gst, holes_of<kB>(a, e_ens));
    } else {
      nbw_birth<R>(ep, ens_of<kB>(a, e_ens), e_rank, gst);
    }
  }
  const unsigned long long nfill = fill_setup<kB>(a, births, s_fb);
  const unsigned long long total = n1 + n0 + nfill;
  for (unsigned long long kk = k0; kk < total; kk += (unsigned long long)gridDim.x * blockDim.x) {
    if (kk == k0 && early != 0) continue;   // taken above
    if (kk < n1) {
      const NcsRec<R> rec = ncslog[kk];
      if (rec.stamp != epoch || a.tile_cnt[1][rec.tile] == 0) continue;
      const int ens = kB ? (int)((rec.species & ~kEvMedium) >> 1) : 0;
      const EnsArgs& E = ens_of<kB>(a, ens);
      const EnsTime tm = time_of<kB>(E);
      const unsigned long long grank = (unsigned long long)a.tile_pre[1][rec.tile] + rec.r_in;
      const unsigned long long rank = kB ? grank - a.map->ev_base[1][ens] : grank;
      const unsigned int* h = holes_of<kB>(a, ens);
      if (rec.species & kEvMedium) brems_event<R>(a, rec, E, tm.step, rank, births, a.flags, gst, h);
      else ncs_event<R>(rec, E, tb, tm.step, rank, births, a.flags, gst, false, 0.0f, h);
    } else if (kk < n1 + n0) {
      nbw_task<R, kB>(a, tb, nbwlog[kk - n1], epoch, gst);
    } else {
      fill_task<R, kB>(a, s_fb, kk - n1 - n0);
    }
  }
  close_step<kB>(a, births);
}


// ======================================================================================
// NCS events with the learned energy sampler (mixed path): a block of 128 threads takes
// 128 logged emissions at a time, evaluates the network for all of them on the tensor
// cores (qed_mlp.cuh), then completes each event as k_events does; the decays and the
// refill tasks follow as in k_events.
// ======================================================================================
template <bool kB>
__global__ void __launch_bounds__(kMlpRows) k_events_mlp(const __grid_constant__ StepArgs a) {
  __shared__ MlpSmem sm;
  __shared__ unsigned int s_fb[kB ? kMaxEns + 1 : 1];
  DevState* gst = a.st;
  const Tabs<float> tb = tabs_global<float>(a.tables);
  // as in k_events: the logs, their extents and the tile counts are final at the start;
  // the sampling runs before the wait for the scan, the births after it
  const unsigned long long nrec = min(gst->cursor[1], a.rec_cap[1]);
  const unsigned long long n0 = min(gst->cursor[0], a.rec_cap[0]);
  const unsigned int epoch = gst->epoch;
  const NcsRec<float>* evlog = reinterpret_cast<const NcsRec<float>*>(a.rec[1]);
  const NbwRec<float>* nbwlog = reinterpret_cast<const NbwRec<float>*>(a.rec[0]);
  const bool births = !(a.flags & (QED_F_NO_RECOIL | QED_F_DROP_PHOTONS));
  // the thread's first decay, up to its pair's birth
  const unsigned long long k0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  bool early = false;
  unsigned int d_tile = 0u, d_rin = 0u, d_ens = 0u;
  NbwPair<float> ep;
  if (k0 < n0) {
    const NbwRec<float> rec = nbwlog[k0];
    if (rec.stamp == epoch && !(rec.ens & kEvMedium)) {
      const EnsArgs& E = ens_of<kB>(a, kB ? (int)rec.ens : 0);
      if (nbw_pair<float>(rec, E, tb, time_of<kB>(E).step, a.tile_cnt[0], &ep)) {
        early = true; d_tile = rec.tile; d_rin = rec.r_in; d_ens = rec.ens;
      }
    }
  }
  const unsigned long long nchunk = (nrec + kMlpRows - 1) / kMlpRows;
  if (blockIdx.x < nchunk) {   // blocks without events skip the tensor-core set-up
  mlp_setup(sm, static_cast<const MlpParams*>(a.mlp));
  unsigned int phase = 0;
  for (unsigned long long c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const unsigned long long kk = c * kMlpRows + threadIdx.x;
    NcsRec<float> rec;
    bool valid = kk < nrec;
    if (valid) {
      rec = evlog[kk];
      valid = rec.stamp == epoch && a.tile_cnt[1][rec.tile] != 0;
    }
    const int ens = valid && kB ? (int)((rec.species & ~kEvMedium) >> 1) : 0;
    const EnsArgs& E = ens_of<kB>(a, ens);
    const EnsTime tm = time_of<kB>(E);
    float x[3] = {0.0f, 0.0f, 0.0f}, lnchi = 0.0f, t = 0.0f;
    if (valid && !(rec.species & kEvMedium)) {
      // the network's inputs: ln chi_e, s = S.zeta, logit of the level uniform
      const SpeciesArgs& L = E.sp[rec.species & 1u];
      const unsigned long long i = rec.i;
      const V3<float> pn = mk<float>(ld<float>(L.px, i), ld<float>(L.py, i), ld<float>(L.pz, i));
      const V3<float> S = mk<float>(ld<float>(L.s1, i), ld<float>(L.s2, i), ld<float>(L.s3, i));
      float pmag = norm(pn);
      pmag = pmag > 0.0f ? pmag : 1e-30f;
      const V3<float> nn = (1.0f / pmag) * pn;
      const V3<float> zeta = cross(nn, mk<float>(rec.ax, rec.ay, rec.az));
      const Uni2 um = uniforms(E.seed, L.id[i], tm.step, 1u);
      double td = log(um.u1) - log1p(-um.u1);
      td = td < kCTLo ? kCTLo : (td > kCTHi ? kCTHi : td);
      t = (float)td;
      lnchi = logf(rec.chi);
      mlp_features(lnchi, dot(S, zeta), t, x);
    }
    bool ok;
    const float y = mlp_rows(sm, x, phase, &ok);
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(&gst->status, QED_STATUS_TIMEOUT);
      break;
    }
    // the emission up to its photon's birth (a bremsstrahlung emission waits whole)
    NcsBirth<float> b;
    bool emitted = false;
    if (valid && !(rec.species & kEvMedium)) {
      // outside the trained chi_e range the table sampler (the fallback) draws the energy
      const bool learned = rec.chi >= kMlpChiLo && rec.chi <= kMlpChiHi;
      emitted = ncs_emit<float>(rec, E, tb, tm.step, births, a.flags, learned, mlp_base(lnchi, t) + 8.0f * y, nullptr,
                                &b);
    }
    pdl_wait();   // returns at once after the first time
    if (valid) {
      const unsigned long long grank = (unsigned long long)a.tile_pre[1][rec.tile] + rec.r_in;
      const unsigned long long rank = kB ? grank - a.map->ev_base[1][ens] : grank;
      const unsigned int* h = holes_of<kB>(a, ens);
      if (rec.species & kEvMedium) brems_event<float>(a, rec, E, tm.step, rank, births, a.flags, gst, h);
      else if (emitted && births) ncs_birth<float>(b, E, rec.species, rank, gst, h);
    }
  }
  mlp_teardown(sm);
  }
  pdl_wait();
  if (early) {
    const int ens = kB ? (int)d_ens : 0;
    unsigned long long rank = (unsigned long long)a.tile_pre[0][d_tile] + d_rin;
    if constexpr (kB) rank -= a.map->ev_base[0][ens];
    nbw_birth<float>(ep, ens_of<kB>(a, ens), rank, gst);
  }
  // the other decays and the refill tasks, as in k_events
  const unsigned long long nfill = fill_setup<kB>(a, births, s_fb);
  for (unsigned long long kk = k0; kk < n0 + nfill; kk += (unsigned long long)gridDim.x * blockDim.x) {
    if (kk == k0 && early) continue;   // taken above
    if (kk < n0) nbw_task<float, kB>(a, tb, nbwlog[kk], epoch, gst);
    else fill_task<float, kB>(a, s_fb, kk - n0);
  }
  close_step<kB>(a, births);
}

// launch with the programmatic-dependent-launch attribute when pdl is set
template <typename... P, typename... A>
inline void launch_k(void (*k)(P...), int grid, int block, cudaStream_t s, bool pdl, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned int)grid);
  cfg.blockDim = dim3((unsigned int)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1u : 0u;
  cudaLaunchKernelEx(&cfg, k, args...);
}

}  // namespace qedk
