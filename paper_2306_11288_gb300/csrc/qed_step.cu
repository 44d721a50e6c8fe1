// qed_step.cu -- the per-step kernels of the spin/polarization-resolved SF-QED hot path
// (Wan et al., arXiv:2306.11288, Secs. II-IV) for sm_103a.
//
// One step = two persistent kernels on the caller's stream:
//   k_photon : gather -> Stokes frame rotation (Eq. rotation) -> VB phase (Eq. rotation2)
//              -> NBW decision (Sec. III D) -> decoupled look-back scan of the decays ->
//              in-place stable compaction of survivors + pair sampling and birth.
//   k_lepton : gather -> Boris (Eqs. boris1-6) -> T-BMT (Eqs. bmt-boris1-4) -> x update
//              -> chi_e -> NCS decision / no-emission spin update / emission (recoil, spin
//              collapse, photon Stokes) -> look-back scan of births -> photon append; the
//              last block to finish updates the live counts and the id counter.
// Tiles of kTile particles are claimed in order from a ticket counter, so the look-back
// only ever waits on tiles already held by running blocks; every wait is bounded and a
// timeout sets QED_STATUS_TIMEOUT instead of hanging.
#include "qed_common.cuh"
#include "qed_internal.h"

namespace qedk {

// ---- memory-order helpers ---------------------------------------------------------
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// look-back word: [epoch:24][flag:2][value:38]; flag 1 = tile aggregate, 2 = inclusive prefix
constexpr int kValBits = 38;
constexpr unsigned long long kValMask = (1ull << kValBits) - 1;

// Warp-parallel look-back, run by all 32 lanes of one warp: publishes this tile's
// aggregate, then inspects 32 predecessors per probe (lane k looks at tile - 1 - k), adds
// the aggregates up to the nearest inclusive prefix, and publishes its own inclusive prefix.
// A predecessor that has not published yet is polled with a bounded number of retries.
__device__ unsigned long long lookback_warp(unsigned long long* words, unsigned int tile, unsigned long long agg,
                                            unsigned int epoch, unsigned int* status) {
  const unsigned int lane = threadIdx.x & 31;
  const unsigned long long ep = (unsigned long long)(epoch & 0xFFFFFFu);
  const unsigned long long tag = ep << 40;
  if (tile == 0) {
    if (lane == 0) st_release(words, tag | (2ull << kValBits) | agg);
    return 0;
  }
  if (lane == 0) st_release(words + tile, tag | (1ull << kValBits) | agg);
  unsigned long long excl = 0;
  long long base = (long long)tile - 1;
  unsigned int spins = 0;
  for (;;) {
    const long long p = base - (long long)lane;
    unsigned int flag = 2;
    unsigned long long v = 0;
    if (p >= 0) {
      const unsigned long long w = ld_acquire(words + p);
      flag = ((w >> 40) == ep) ? (unsigned int)((w >> kValBits) & 3ull) : 0u;
      v = w & kValMask;
    }
    const unsigned int ready = __ballot_sync(0xffffffffu, flag != 0);
    const unsigned int pmask = __ballot_sync(0xffffffffu, flag == 2);
    const unsigned int first = pmask ? (unsigned int)(__ffs(pmask) - 1) : 31u;
    const unsigned int need = first == 31u ? 0xffffffffu : ((2u << first) - 1u);
    if ((ready & need) != need) {
      if (++spins > (1u << 22)) {   // about a second: give up, flag it, never hang
        if (lane == 0) atomicOr(status, QED_STATUS_TIMEOUT);
        break;
      }
      __nanosleep(32);
      continue;
    }
    unsigned long long mine = (lane <= first) ? v : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    excl += mine;
    if (pmask) break;
    base -= 32;
  }
  if (lane == 0) st_release(words + tile, tag | (2ull << kValBits) | ((excl + agg) & kValMask));
  return excl;
}

// block-wide exclusive scan of one flag per thread + decoupled look-back across tiles.
// Returns this thread's global rank among flagged threads; *tile_total = flags in tile.
struct ScanShared {
  unsigned int warp_off[kTile / 32];
  unsigned long long prefix;
  unsigned int total;
};

__device__ __forceinline__ unsigned long long block_rank(bool flag, unsigned int tile, unsigned long long* words,
                                                         unsigned int epoch, unsigned int* status, ScanShared& sh,
                                                         unsigned int* tile_total) {
  const unsigned int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int ballot = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) sh.warp_off[warp] = __popc(ballot);
  __syncthreads();
  if (warp == 0) {
    constexpr unsigned int nw = kTile / 32;
    const unsigned int mine = lane < nw ? sh.warp_off[lane] : 0u;
    unsigned int c = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int v = __shfl_up_sync(0xffffffffu, c, o);
      if (lane >= (unsigned)o) c += v;
    }
    const unsigned int total = __shfl_sync(0xffffffffu, c, 31);
    if (lane < nw) sh.warp_off[lane] = c - mine;
    const unsigned long long pre = lookback_warp(words, tile, total, epoch, status);
    if (lane == 0) {
      sh.prefix = pre;
      sh.total = total;
    }
  }
  __syncthreads();
  *tile_total = sh.total;
  return sh.prefix + sh.warp_off[warp] + __popc(ballot & ((1u << lane) - 1u));
}

// ---- external fields (paper Sec. II D) ---------------------------------------------
template <typename R>
struct EB { V3<R> E, B; };

__device__ __forceinline__ double reduce_2pi(double ph) {
  return ph - 6.283185307179586477 * rint(ph * 0.15915494309189533577);
}

template <typename R>
__device__ __forceinline__ R tsc_gather(const float* g, int nx, int ny, double X, double Y) {
  const double fx = floor(X + 0.5), fy = floor(Y + 0.5);
  const int ig = (int)fx, jg = (int)fy;
  const R dx = (R)(X - fx), dy = (R)(Y - fy);
  const R wx[3] = {R(0.5) * (R(0.5) - dx) * (R(0.5) - dx), R(0.75) - dx * dx, R(0.5) * (R(0.5) + dx) * (R(0.5) + dx)};
  const R wy[3] = {R(0.5) * (R(0.5) - dy) * (R(0.5) - dy), R(0.75) - dy * dy, R(0.5) * (R(0.5) + dy) * (R(0.5) + dy)};
  R acc = R(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int j = jg - 1 + b;
    if (j < 0 || j >= ny) continue;
    R row = R(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int i = ig - 1 + c;
      if (i < 0 || i >= nx) continue;
      row += wx[c] * (R)__ldg(g + (size_t)j * nx + i);
    }
    acc += wy[b] * row;
  }
  return acc;
}

template <typename R>
__device__ __forceinline__ EB<R> gather(const qed_fields& f, double x, double y, double z, double t) {
  EB<R> r;
  r.E = mk<R>(0, 0, 0);
  r.B = mk<R>(0, 0, 0);
  if (f.kind == QED_FIELD_UNIFORM) {
    r.E = mk<R>((R)f.E[0], (R)f.E[1], (R)f.E[2]);
    r.B = mk<R>((R)f.B[0], (R)f.B[1], (R)f.B[2]);
  } else if (f.kind == QED_FIELD_PLANE || f.kind == QED_FIELD_GAUSS) {
    const double phi = t + z;
    const double s = (phi - f.phi0) / f.len;
    if (s < 0.0 || s > 1.0) return r;
    R sn, cs;
    m_sincos((R)(kPi * s), &sn, &cs);
    R g = (R)f.a0 * sn * sn;
    R ph = (R)reduce_2pi(phi);
    if (f.kind == QED_FIELD_GAUSS) {
      const R zeta = (R)(f.zf - z);
      const R zr = (R)(0.5 * f.w0 * f.w0);
      const R q = zeta / zr;
      const R w0 = (R)f.w0;
      const R w2 = w0 * w0 * (R(1) + q * q);
      const R r2 = (R)(x * x + y * y);
      g = g * (w0 / sqrt(w2)) * m_exp(-r2 / w2);
      ph = ph - R(0.5) * r2 * zeta / (zeta * zeta + zr * zr) + m_atan(q);
    }
    R sp, cp;
    m_sincos(ph, &sp, &cp);
    r.E.x = g * cp;
    r.E.y = f.circular ? g * sp : R(0);
    r.B.x = r.E.y;
    r.B.y = -r.E.x;
  } else if (f.kind == QED_FIELD_GRID2D) {
    const double X = (x - f.x0) / f.dx, Y = (y - f.y0) / f.dy;
    r.E.x = tsc_gather<R>(f.gEx, f.nx, f.ny, X - 0.5, Y);
    r.E.y = tsc_gather<R>(f.gEy, f.nx, f.ny, X, Y - 0.5);
    r.E.z = tsc_gather<R>(f.gEz, f.nx, f.ny, X, Y);
    r.B.x = tsc_gather<R>(f.gBx, f.nx, f.ny, X, Y - 0.5);
    r.B.y = tsc_gather<R>(f.gBy, f.nx, f.ny, X - 0.5, Y);
    r.B.z = tsc_gather<R>(f.gBz, f.nx, f.ny, X - 0.5, Y - 0.5);
  }
  return r;
}

// canonical transverse frame of n: e1 = unit(y x n) (unit(n x x) near +-y), e2 = n x e1
template <typename R>
__device__ __forceinline__ void frame(V3<R> n, V3<R>& e1, V3<R>& e2) {
  R a = n.z, b = R(0), c = -n.x;
  R m2 = a * a + c * c;
  if (m2 < R(1e-20)) { a = R(0); b = n.z; c = -n.y; m2 = b * b + c * c; }
  const R inv = R(1) / sqrt(m2);
  e1 = mk<R>(a * inv, b * inv, c * inv);
  e2 = cross(n, e1);
}

// ---- table access --------------------------------------------------------------------
template <typename R>
struct Tabs {
  const R* g;     // full table block in global memory
  const R* s;     // shared-memory copy of the 1-D rate tables (starts at kOffRA)
  __device__ __forceinline__ void ncs_rates(R chi, R& A, R& B) const {
    const R X = (m_log(chi) - R(kRLo)) * R((kNR - 1) / (kRHi - kRLo));
    A = chi * lagrange4(s, kNR, X);
    B = chi * lagrange4(s + kNR, kNR, X);
  }
  __device__ __forceinline__ R ncs_inv(int comp, R chi, R t) const {
    const R X = (m_log(chi) - R(kRLo)) * R((kNCX - 1) / (kRHi - kRLo));
    const R ht = R((kCTHi - kCTLo) / (kNCT - 1));
    const size_t o = (size_t)comp * kNCX * kNCT;
    return table2d(g + kOffCY + o, g + kOffCD + o, kNCX, kNCT, X, (t - R(kCTLo)) / ht, ht);
  }
  __device__ __forceinline__ void nbw_rates(R chig, R& T0, R& T3) const {
    const R X = (m_log(chig) - R(kBLo)) * R((kNBX - 1) / (kBHi - kBLo));
    const R damp = m_exp(R(-8.0 / 3.0) / chig);
    T0 = damp * lagrange4(s + (kOffT0 - kOffRA), kNBX, X);
    T3 = damp * lagrange4(s + (kOffT3 - kOffRA), kNBX, X);
  }
  __device__ __forceinline__ R nbw_inv(int comp, R chig, R t) const {
    const R X = (m_log(chig) - R(kBLo)) * R((kNBX - 1) / (kBHi - kBLo));
    const R ht = R((kBTHi - kBTLo) / (kNBT - 1));
    const size_t o = (size_t)comp * kNBX * kNBT;
    return table2d(g + kOffBY + o, g + kOffBD + o, kNBX, kNBT, X, (t - R(kBTLo)) / ht, ht);
  }
  __device__ __forceinline__ void vb_m(R chig, R& mp, R& mq) const {
    if (chig < R(kVbMin)) { mp = R(4); mq = R(7); return; }
    const R X = (m_log(chig) - R(kVLo)) * R((kNV - 1) / (kVHi - kVLo));
    mp = lagrange4(s + (kOffMP - kOffRA), kNV, X);
    mq = lagrange4(s + (kOffMQ - kOffRA), kNV, X);
  }
  __device__ __forceinline__ void k(R x, R& k13, R& k23, R& ik) const { kfun(g, x, k13, k23, ik); }
};

template <typename R>
__device__ __forceinline__ void stage_rates(const R* g, R* s) {
  for (int i = threadIdx.x; i < (int)kSmemRateLen; i += blockDim.x) s[i] = g[kOffRA + i];
}

template <typename T>
__device__ __forceinline__ T ld(const void* p, unsigned long long i) { return reinterpret_cast<const T*>(p)[i]; }
template <typename T>
__device__ __forceinline__ void stv(void* p, unsigned long long i, T v) { reinterpret_cast<T*>(p)[i] = v; }

__device__ __forceinline__ void count_event(unsigned long long* ctr, bool flag) {
  const unsigned int b = __ballot_sync(0xffffffffu, flag);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(ctr, (unsigned long long)__popc(b));
}

// ======================================================================================
// photon kernel
// ======================================================================================
// resident blocks per SM requested from the register allocator
template <typename R> struct Occ { static constexpr int v = sizeof(R) == 4 ? 3 : 2; };

template <typename R>
__global__ void __launch_bounds__(kTile, Occ<R>::v) k_photon(StepArgs a) {
  __shared__ R s_rates[kSmemRateLen];
  __shared__ ScanShared s_scan;
  __shared__ unsigned int s_tile;
  DevState* st = a.st;
  const Tabs<R> tb{reinterpret_cast<const R*>(a.tables), s_rates};
  stage_rates(tb.g, s_rates);
  const SpeciesArgs& P = a.sp[2];
  const unsigned long long n = P.present ? st->n_live[2] : 0ull;
  const unsigned int ntiles = (unsigned int)((n + kTile - 1) / kTile);
  const unsigned int epoch = st->epoch;
  const unsigned long long ne0 = st->n_live[0], np0 = st->n_live[1];
  const unsigned long long id0 = st->next_id;
  const R dt = (R)a.dt;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(&st->ticket[0], 1u);
    __syncthreads();
    const unsigned int tile = s_tile;
    if (tile >= ntiles) break;
    const unsigned long long i = (unsigned long long)tile * kTile + threadIdx.x;
    const bool live = i < n;
    double x = 0, y = 0, z = 0;
    V3<R> k = mk<R>(1, 0, 0), xi = mk<R>(0, 0, 0);
    R th = 0, wgt = 0;
    uint64_t id = 0;
    // everything is loaded before the scan: after it, compaction may overwrite any slot
    if (live) {
      x = P.x[i]; y = P.y[i]; z = P.z[i];
      k = mk<R>(ld<R>(P.px, i), ld<R>(P.py, i), ld<R>(P.pz, i));
      xi = mk<R>(ld<R>(P.s1, i), ld<R>(P.s2, i), ld<R>(P.s3, i));
      th = ld<R>(P.theta, i);
      wgt = ld<R>(P.w, i);
      id = P.id[i];
    }
    bool decay = false, range = false;
    R om = norm(k);
    const V3<R> nn = (R(1) / om) * k;
    V3<R> P1 = mk<R>(0, 0, 0), P2 = mk<R>(0, 0, 0);
    R chig = 0, T0 = 0, T3 = 0, rmix = 0;
    if (live && (a.flags & (QED_F_VB | QED_F_NBW))) {
      const EB<R> f = gather<R>(a.f, x, y, z, a.t);
      const R ne = dot(nn, f.E);
      const V3<R> Er = f.E - ne * nn + cross(nn, f.B);
      const R er = norm(Er);
      if (er > R(0)) {
        chig = R(kXiL) * om * er;
        P1 = (R(1) / er) * Er;
        P2 = cross(nn, P1);
        V3<R> e1, e2;
        frame(nn, e1, e2);
        const R thn = m_atan2(dot(P1, e2), dot(P1, e1));
        R s2, c2;
        m_sincos(R(2) * (thn - th), &s2, &c2);
        const R x1 = xi.x * c2 - xi.z * s2, x3 = xi.x * s2 + xi.z * c2;
        xi.x = x1; xi.z = x3;
        th = thn;
        if (a.flags & QED_F_VB) {
          R mp, mq;
          tb.vb_m(chig > R(kVbMax) ? R(kVbMax) : chig, mp, mq);
          const R dphi = (mp - mq) * R(kAlpha / (90.0 * kPi) * kXiL) * om * er * er * dt;
          R sd, cd;
          m_sincos(dphi, &sd, &cd);
          const R y1 = cd * xi.x - sd * xi.y, y2 = sd * xi.x + cd * xi.y;
          xi.x = y1; xi.y = y2;
        }
        if ((a.flags & QED_F_NBW) && om >= R(2) && chig >= R(kChigMin)) {
          if (chig > R(kChigMax)) { chig = R(kChigMax); range = true; }
          tb.nbw_rates(chig, T0, T3);
          const R Pd = R(kAlpha / (1.7320508075688772935 * kPi * kXiL)) / om * (T0 - xi.z * T3) * dt;
          const Uni2 u = uniforms(a.seed, id, a.step, 3u);
          decay = u.u0 < (double)Pd;
          rmix = (R)u.u1;
        }
      }
    }
    count_event(&st->ev[3], range);
    unsigned int tile_dec;
    const unsigned long long rank = block_rank(live && decay, tile, a.look[0], epoch, &st->status, s_scan, &tile_dec);
    if (live && !decay) {
      const unsigned long long out = i - rank;   // decays before i
      P.x[out] = x + a.dt * (double)nn.x;
      P.y[out] = y + a.dt * (double)nn.y;
      P.z[out] = z + a.dt * (double)nn.z;
      stv<R>(P.s1, out, xi.x); stv<R>(P.s2, out, xi.y); stv<R>(P.s3, out, xi.z);
      stv<R>(P.theta, out, th);
      if (out != i) {
        stv<R>(P.px, out, k.x); stv<R>(P.py, out, k.y); stv<R>(P.pz, out, k.z);
        stv<R>(P.w, out, wgt);
        P.id[out] = id;
      }
    }
    if (live && decay) {
      // ---- pair: energy split (mixture over xi3' = +-1), spins (Sec. III D) ----------
      const Uni2 u2 = uniforms(a.seed, id, a.step, 4u);
      const R w0 = R(0.5) * (R(1) + xi.z) * (T0 - T3);
      const int comp = (rmix * (T0 - xi.z * T3) < w0) ? 0 : 1;
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
      // joint probabilities of (s+, s-) in {++, +-, -+, --} from Eqs. G0-G3 (W0/2 dropped)
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
      for (int q = 0; q < 4; ++q) {
        acc += pk[q];
        if (o == 3 && q < 3 && rr < acc) o = q;
      }
      const R sp = (o < 2) ? R(1) : R(-1), sm = (o % 2 == 0) ? R(1) : R(-1);
      const R pp = sqrt(ep * ep - R(1)), pm = sqrt(em * em - R(1));
      const SpeciesArgs* dst[2] = {&a.sp[0], &a.sp[1]};
      const unsigned long long base[2] = {ne0, np0};
      const R pmag[2] = {pm, pp};
      const V3<R> spin[2] = {sm * Sm, sp * Sp};
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const SpeciesArgs& L = *dst[s];
        const unsigned long long j = base[s] + rank;
        if (!L.present || j >= L.cap) {
          atomicOr(&st->status, QED_STATUS_CAPACITY);
          atomicAdd(&st->ev[4], 1ull);
          continue;
        }
        L.x[j] = x; L.y[j] = y; L.z[j] = z;
        stv<R>(L.px, j, pmag[s] * nn.x); stv<R>(L.py, j, pmag[s] * nn.y); stv<R>(L.pz, j, pmag[s] * nn.z);
        stv<R>(L.s1, j, spin[s].x); stv<R>(L.s2, j, spin[s].y); stv<R>(L.s3, j, spin[s].z);
        stv<R>(L.w, j, wgt);
        L.id[j] = id0 + 2ull * rank + (unsigned long long)s;
      }
    }
    if (tile == ntiles - 1 && threadIdx.x == 0) {
      const unsigned long long ndec = s_scan.prefix + tile_dec;
      st->n_nbw = ndec;
      st->n_surv = n - ndec;
      st->ev[2] += ndec;
    }
  }
}

// ======================================================================================
// lepton kernel
// ======================================================================================
template <typename R>
__global__ void __launch_bounds__(kTile, Occ<R>::v) k_lepton(StepArgs a) {
  __shared__ R s_rates[kSmemRateLen];
  __shared__ ScanShared s_scan;
  __shared__ unsigned int s_tile;
  DevState* st = a.st;
  const Tabs<R> tb{reinterpret_cast<const R*>(a.tables), s_rates};
  stage_rates(tb.g, s_rates);
  const unsigned long long n0 = a.sp[0].present ? st->n_live[0] : 0ull;
  const unsigned long long n1 = a.sp[1].present ? st->n_live[1] : 0ull;
  const unsigned int t0 = (unsigned int)((n0 + kTile - 1) / kTile);
  const unsigned int ntiles = t0 + (unsigned int)((n1 + kTile - 1) / kTile);
  const unsigned int epoch = st->epoch;
  const unsigned long long nsurv = st->n_surv, nnbw = st->n_nbw;
  const unsigned long long id0 = st->next_id + 2ull * nnbw;
  const SpeciesArgs& G = a.sp[2];
  const R dt = (R)a.dt;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(&st->ticket[1], 1u);
    __syncthreads();
    const unsigned int tile = s_tile;
    if (tile >= ntiles) break;
    const int sp_idx = tile < t0 ? 0 : 1;
    const SpeciesArgs& L = a.sp[sp_idx];
    const unsigned long long nsp = sp_idx == 0 ? n0 : n1;
    const unsigned long long i = (unsigned long long)(tile - (sp_idx == 0 ? 0u : t0)) * kTile + threadIdx.x;
    const bool live = i < nsp;
    const R q = sp_idx == 0 ? R(-1) : R(1);
    double x = 0, y = 0, z = 0;
    V3<R> p = mk<R>(0, 0, 1), S = mk<R>(0, 1, 0);
    uint64_t id = 0;
    if (live) {
      x = L.x[i]; y = L.y[i]; z = L.z[i];
      p = mk<R>(ld<R>(L.px, i), ld<R>(L.py, i), ld<R>(L.pz, i));
      S = mk<R>(ld<R>(L.s1, i), ld<R>(L.s2, i), ld<R>(L.s3, i));
      id = L.id[i];
    }
    bool emit = false, range = false;
    V3<R> kph = mk<R>(0, 0, 0), xiph = mk<R>(0, 0, 0);
    R thph = 0;
    if (live) {
      const EB<R> f = gather<R>(a.f, x, y, z, a.t);
      // Boris push
      const R hq = R(0.5) * q * dt;
      const V3<R> pm = p + hq * f.E;
      const R gm = sqrt(R(1) + dot(pm, pm));
      const V3<R> tau = (hq / gm) * f.B;
      const V3<R> pp = pm + cross(pm, tau);
      const V3<R> sig = (R(2) / (R(1) + dot(tau, tau))) * tau;
      V3<R> pn = pm + cross(pp, sig) + hq * f.E;
      // T-BMT with beta, gamma of the mean of p^{n-1/2} and p^{n+1/2}
      if (a.flags & QED_F_SPIN) {
        const V3<R> pa = R(0.5) * (p + pn);
        const R ga = sqrt(R(1) + dot(pa, pa));
        const V3<R> be = (R(1) / ga) * pa;
        const R gg = ga / (ga + R(1));
        const V3<R> Om = (-R(kAe) * gg * dot(be, f.B)) * be + (R(kAe) + R(1) / ga) * f.B +
                         (-(R(kAe) + R(1) / (ga + R(1)))) * cross(be, f.E);
        const V3<R> tv = hq * Om;
        const V3<R> ov = (R(2) / (R(1) + dot(tv, tv))) * tv;
        const V3<R> S1 = S + cross(S, tv);
        S = S + cross(S1, ov);
      }
      const R g1 = sqrt(R(1) + dot(pn, pn));
      x += a.dt * (double)(pn.x / g1);
      y += a.dt * (double)(pn.y / g1);
      z += a.dt * (double)(pn.z / g1);
      if (a.flags & QED_F_NCS) {
        R pmag = norm(pn);
        pmag = pmag > R(0) ? pmag : R(1e-30);
        const V3<R> nn = (R(1) / pmag) * pn;
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
        const R vm = sqrt(vm2);
        R chi = R(kXiL) * sqrt(vm2 + nE * nE);
        if (chi >= R(kChiMin) && vm > R(0)) {
          if (chi > R(kChiMax)) { chi = R(kChiMax); range = true; }
          const V3<R> av = (q / vm) * v;    // unit acceleration direction
          const V3<R> zeta = cross(nn, av);
          R A, B;
          tb.ncs_rates(chi, A, B);
          const R s = dot(S, zeta);
          const R pref = R(kAlpha / (1.7320508075688772935 * kPi * kXiL)) / g1;
          const R Wa = pref * A, Wb = pref * B;
          const R Pe = (Wa - s * Wb) * dt;
          const Uni2 u = uniforms(a.seed, id, a.step, 0u);
          if (u.u0 < (double)Pe) {
            emit = true;
            const Uni2 um = uniforms(a.seed, id, a.step, 1u);
            const Uni2 us = uniforms(a.seed, id, a.step, 2u);
            // photon energy fraction: two-component mixture at s = S.zeta (Eq. Wspin2)
            const R wplus = R(0.5) * (R(1) + s) * (A - B);
            const int comp = ((R)um.u0 * (A - s * B) < wplus) ? 0 : 1;
            const double l = um.u1;
            R tt;
            if (sizeof(R) == 8) tt = (R)(log(l) - log1p(-l));
            else tt = m_log((R)l) - m_log((R)(1.0 - l));
            tt = tt < R(kCTLo) ? R(kCTLo) : (tt > R(kCTHi) ? R(kCTHi) : tt);
            const R uu = m_exp(tb.ncs_inv(comp, chi, tt));
            const R omr = R(1) / (R(1) + uu), rr = uu * omr;
            const R om = rr * g1;
            // spin collapse along the SQA of Eq. F0 (linear in S_f: c0 + g.S_f)
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
            // photon Stokes: pure states +-F/|F| from Eqs. F1-F3 at (S_i, S_f)
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
            if (fm > R(0)) {
              const R sg = ((R)us.u1 < R(0.5) * (R(1) + fm / F0)) ? R(1) : R(-1);
              xiph = mk<R>(sg * F1 / fm, sg * F2 / fm, sg * F3 / fm);
            }
            S = Sf;
            if (!(a.flags & QED_F_NO_RECOIL)) {
              // recoil p_f = p_i - omega n, |p_f| = (1-r) gamma - (gamma - |p|)
              const R pf = omr * g1 - R(1) / (g1 + pmag);
              pn = pf * nn;
              kph = om * nn;
              V3<R> e1, e2;
              frame(nn, e1, e2);
              thph = m_atan2(dot(av, e2), dot(av, e1));
            }
          } else {
            // no emission: posterior mean spin, then collapse with P(+) = (1+|S|)/2
            const R den = R(1) / (R(1) - Pe);
            const V3<R> Sb = (den * (R(1) - Wa * dt)) * S + (den * Wb * dt) * zeta;
            const R m = norm(Sb);
            const R sg = ((R)u.u1 < R(0.5) * (R(1) + m)) ? R(1) : R(-1);
            S = (sg / m) * Sb;
          }
        }
      }
      p = pn;
      L.x[i] = x; L.y[i] = y; L.z[i] = z;
      stv<R>(L.px, i, p.x); stv<R>(L.py, i, p.y); stv<R>(L.pz, i, p.z);
      stv<R>(L.s1, i, S.x); stv<R>(L.s2, i, S.y); stv<R>(L.s3, i, S.z);
    }
    count_event(&st->ev[sp_idx], emit);
    count_event(&st->ev[3], range);
    const bool birth = live && emit && !(a.flags & (QED_F_NO_RECOIL | QED_F_DROP_PHOTONS));
    unsigned int tile_b;
    const unsigned long long rank = block_rank(birth, tile, a.look[1], epoch, &st->status, s_scan, &tile_b);
    if (birth) {
      const unsigned long long j = nsurv + rank;
      if (!G.present || j >= G.cap) {
        atomicOr(&st->status, QED_STATUS_CAPACITY);
        atomicAdd(&st->ev[4], 1ull);
      } else {
        G.x[j] = x; G.y[j] = y; G.z[j] = z;
        stv<R>(G.px, j, kph.x); stv<R>(G.py, j, kph.y); stv<R>(G.pz, j, kph.z);
        stv<R>(G.s1, j, xiph.x); stv<R>(G.s2, j, xiph.y); stv<R>(G.s3, j, xiph.z);
        stv<R>(G.theta, j, thph);
        stv<R>(G.w, j, ld<R>(L.w, i));
        G.id[j] = id0 + rank;
      }
    }
    if (tile == ntiles - 1 && threadIdx.x == 0) st->n_ncs_tot = s_scan.prefix + tile_b;
  }
  // the last block to finish closes the step: counts, id counter, statistics, resets
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int d = atomicAdd(&st->done[1], 1u);
    if (d == gridDim.x - 1) {
      __threadfence();
      volatile DevState* v = st;
      const unsigned long long nbw = v->n_nbw, ncs = v->n_ncs_tot, surv = v->n_surv;
      for (int s = 0; s < 2; ++s) {
        if (!a.sp[s].present) continue;
        unsigned long long nn = v->n_live[s] + nbw;
        v->n_live[s] = nn > a.sp[s].cap ? a.sp[s].cap : nn;
      }
      if (G.present) {
        const unsigned long long nn = surv + ncs;
        v->n_live[2] = nn > G.cap ? G.cap : nn;
      }
      v->next_id = v->next_id + 2ull * nbw + ncs;
      if (a.user_stats) {
        a.user_stats->n_ncs[0] += v->ev[0];
        a.user_stats->n_ncs[1] += v->ev[1];
        a.user_stats->n_nbw += v->ev[2];
        a.user_stats->n_range += v->ev[3];
        a.user_stats->n_drop += v->ev[4];
        a.user_stats->n_steps += 1;
      }
      if (v->ev[3]) v->status |= QED_STATUS_TABLE_RANGE;
      for (int k = 0; k < 6; ++k) v->ev[k] = 0;
      v->n_nbw = 0; v->n_surv = 0; v->n_ncs_tot = 0;
      v->ticket[0] = 0; v->ticket[1] = 0;
      v->done[0] = 0; v->done[1] = 0;
      v->epoch = v->epoch + 1;
      __threadfence();
    }
  }
}

template <typename R>
static qed_status launch_t(const StepArgs& a, int nph, int nlep, cudaStream_t s, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], s);
  k_photon<R><<<nph, kTile, 0, s>>>(a);
  if (ev) cudaEventRecord(ev[1], s);
  k_lepton<R><<<nlep, kTile, 0, s>>>(a);
  if (ev) cudaEventRecord(ev[2], s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("step launch failed: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  return QED_OK;
}

qed_status launch_step(const StepArgs& a, qed_precision prec, int nph, int nlep, cudaStream_t s, cudaEvent_t* ev) {
  return prec == QED_PREC_F64 ? launch_t<double>(a, nph, nlep, s, ev) : launch_t<float>(a, nph, nlep, s, ev);
}

qed_status step_grid_sizes(qed_precision prec, int* nph, int* nlep) {
  int dev = 0, sms = 0, b0 = 0, b1 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (prec == QED_PREC_F64) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_photon<double>, kTile, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_lepton<double>, kTile, 0);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_photon<float>, kTile, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_lepton<float>, kTile, 0);
  }
  if (e != cudaSuccess || b0 < 1 || b1 < 1) {
    set_error("occupancy query failed: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  *nph = sms * b0;
  *nlep = sms * b1;
  return QED_OK;
}

}  // namespace qedk
