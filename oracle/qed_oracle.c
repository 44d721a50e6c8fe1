/*
 * qed_oracle.c -- FP64 CPU oracle of the spin/polarization-resolved SF-QED step of
 * Wan et al., arXiv:2306.11288.  TEST INFRASTRUCTURE ONLY (see qed_oracle.h).
 *
 * Plain, slow, compiled with -ffp-contract=off; single-threaded unless or_set_threads asks
 * for an OpenMP loop over the particles of a step (each particle's outcome goes to its own
 * slot and births are appended in index order afterwards, so the results do not depend on
 * the thread count).  Every function
 * names the passage of the paper it follows.  Where the paper is silent, garbled or
 * self-contradictory, the reading taken is stated at the point of use; the full list
 * is in the repository's design notes ("readings").
 *
 * Parity pins (tests/test_oracle_*.py):
 *   Philox4x32-10 ......... Random123 known-answer vectors
 *   K_nu, IntK ............ scipy.special.kve / quad, DLMF closed forms
 *   Scorer Gi' ............ mpmath.scorergi (numerical derivative)
 *   tables ................ off-grid brute-force quadrature (scipy)
 *   rate algebra .......... Eq. NCSW -> Wspin -> Wspin2 -> unpolarised; Eq. BW ->
 *                           BW_pos / BWeleAxis -> BWprob; positivity
 *   NCS normalisation ..... classical radiated power (Sec. III A, Eq. for F_RR,cl)
 *   NBW normalisation ..... small-chi_gamma Laplace asymptote
 *   VB .................... M -> 4, 7 as chi_gamma -> 0 (Eq. eqn26)
 *   Boris ................. |p| conserved in pure B; plane-wave invariants
 *   T-BMT ................. g-2 precession closed form
 *   spin MC ............... mean one-step drift = radiative T-BMT (Eq. spin1)
 *   radiative pusher ...... q, psi1..3 vs scipy quadrature and Mellin small-chi forms;
 *                           one LL step radiates the Larmor power; Sokolov-Ternov
 *                           build-up; MC mean = MLL + radiative T-BMT (Sec. III C)
 *   field models .......... B = k x E; the paraxial Gaussian satisfies the paraxial wave
 *                           equation of a beam along -z, is flat and Gaussian at its
 *                           focus, carries the same transverse power at every z, and
 *                           keeps |E_perp| constant when circular
 *   sharded ids ........... or_shard_bases against its closed form for three ranks (the
 *                           id blocks tile the range); decide + commit = or_step; two
 *                           ranks = one process stepping the population in rank order
 */
#include "qed_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- constants (CODATA 2018; the paper fixes none of them) ------------------- */
static const double OR_PI = 3.14159265358979323846;
static const double OR_ALPHA = 7.2973525693e-3;     /* fine-structure constant   */
static const double OR_XIL = 2.42631023867e-6;      /* hbar w0/(m c^2), lambda=1um */
static const double OR_AE = 1.15965218128e-3;       /* g/2 - 1 of the electron   */
static const double OR_CHI_MIN = 1e-4, OR_CHI_MAX = 1e3;     /* chi_e range        */
static const double OR_CHIG_MIN = 1e-2, OR_CHIG_MAX = 1e3;   /* chi_gamma, NBW     */
static const double OR_VB_MIN = 1e-3, OR_VB_MAX = 1e3;       /* chi_gamma, VB      */
/* classical electron radius (CODATA 2018, 2.8179403262e-15 m) in units of 1/k0 = 1 um/(2 pi) */
#define OR_R0N (2.8179403262e-9 * 2.0 * 3.14159265358979323846)

/* ---- table grids (a specification both implementations follow) -------------- */
#define NK 1024
#define K_LO (-6.907755278982137)   /* ln 1e-3 */
#define K_HI (11.512925464970229)   /* ln 1e5  */
#define NR 512
#define R_LO (-9.210340371976182)   /* ln 1e-4 */
#define R_HI (6.907755278982137)    /* ln 1e3  */
#define NCX 256
#define NCT 512
#define CT_LO (-38.0)
#define CT_HI (38.0)
#define NBX 256
#define B_LO (-4.605170185988091)   /* ln 1e-2 */
#define B_HI (6.907755278982137)
#define NBT 256
#define BT_LO (-38.0)
#define BT_HI (0.0)
#define NV 1024
#define V_LO (-6.907755278982137)
#define V_HI (6.907755278982137)
#define NMG 256                        /* medium tables: energy rows, ln E on [ln 2, ln 2e6] */
#define MG_LO 0.69314718055994531    /* ln 2 */
#define MG_HI 14.508657738524219     /* ln 2e6 */
#define NMS 512                        /* medium tables: cumulative nodes in s on [0, 1]     */

struct or_ctx {
  double kv[3][NK], kd[3][NK];                  /* scaled K13, K23, IntK13 + d/dlnx */
  double ra[NR], rb[NR];                        /* A/chi, B/chi                  */
  double cy[2][NCX][NCT], cd[2][NCX][NCT];      /* NCS inverse CDF: ln u, d/dt    */
  double t0s[NBX], t3s[NBX];                    /* T0, T3 times exp(8/(3chi_g))   */
  double by[2][NBX][NBT], bd[2][NBX][NBT];      /* NBW half inverse CDF: ln delta */
  double mpar[NV], mperp[NV];                   /* VB M_par, M_perp               */
  double rr[4][NR];                             /* q, psi1/chi^3, psi2/chi^3, psi3/chi^3 */
  uint64_t next_id;
  int has_medium;                               /* bremsstrahlung / pair tables present  */
  or_medium med;
  double mb[NMG][NMS], mp[NMG][NMS];            /* cumulative brems (y) and pair (x) cross-sections */
  double near_tol;                              /* log decisions with |r - thr| < near_tol thr */
  int threads;                                  /* particle-loop threads of or_step (OpenMP) */
  uint64_t nlog, logcap;
  uint64_t *log_id; uint32_t *log_step, *log_kind; double *log_margin;
  /* a step decided by or_step_decide and not yet committed: the decayed photons' slots
     (index order), the pairs they create, the photons the leptons emit (e- then e+) */
  int pending;
  void *p_be, *p_bp, *p_bg;
  uint64_t *p_dec, p_nnbw, p_nncs, p_nncs_e;
};

/* ======================================================================= *
 *  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the   *
 *  published round function: two 32x32->64 products, Weyl key schedule. *
 * ======================================================================= */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* two uniforms in [0,1) with 53 random bits each from one Philox block;
 * counter = (id_lo, id_hi, step, ctr), key = seed */
void or_uniforms(uint64_t seed, uint64_t id, uint32_t step, uint32_t ctr, double u[2]) {
  uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, ctr};
  uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  or_philox4x32_10(c, k, o);
  const double two_m53 = 1.0 / 9007199254740992.0;
  u[0] = (double)(((uint64_t)(o[0] >> 5) << 26) + (o[1] >> 6)) * two_m53;
  u[1] = (double)(((uint64_t)(o[2] >> 5) << 26) + (o[3] >> 6)) * two_m53;
}

/* ======================================================================= *
 *  Modified Bessel functions (the paper's K_1/3, K_2/3, IntK_1/3 of      *
 *  Eqs. F0-F3, G0-G3).  DLMF 10.32.9: K_nu(x) = int_0^inf e^{-x cosh t}   *
 *  cosh(nu t) dt; integrating in x gives IntK_nu(x) = int_0^inf           *
 *  e^{-x cosh t} cosh(nu t)/cosh t dt.  Trapezoid rule in t (exponential  *
 *  convergence for these entire integrands).  Returns e^x times each.     *
 * ======================================================================= */
void or_besselk_scaled(double x, double out[3]) {
  double h = 0.05;
  double hx = 0.5 / sqrt(x);
  if (hx < h) h = hx;
  double s13 = 0.5, s23 = 0.5, si = 0.5;   /* t = 0 term, weight 1/2 */
  for (int k = 1; k < 200000; ++k) {
    double t = k * h;
    double ch = cosh(t);
    double e = exp(-x * (ch - 1.0));
    double a = e * cosh(t / 3.0);
    double b = e * cosh(2.0 * t / 3.0);
    s13 += a; s23 += b; si += a / ch;
    if (x * (ch - 1.0) > 1.0 && b < 1e-18 * s23) break;
  }
  out[0] = h * s13; out[1] = h * s23; out[2] = h * si;
}

/* ---- the K-table: cubic Hermite in ln x with exact derivatives ------------- */
/* small-x form below the table (two terms of each I_{+-nu} power series):
 * K_nu = pi/(2 sin(nu pi)) [I_{-nu} - I_nu], IntK13 = pi/sqrt3 - int_0^x K13 */
static void or_k_small(double x, double out[3]) {
  const double g13 = 2.678938534707747633;   /* Gamma(1/3) */
  const double g23 = 1.354117939426400417;   /* Gamma(2/3) */
  const double g43 = g13 / 3.0, g53 = 2.0 * g23 / 3.0;
  const double g73 = 4.0 * g43 / 3.0, g83 = 5.0 * g53 / 3.0;
  const double c = OR_PI / (2.0 * sin(OR_PI / 3.0));  /* same for nu = 1/3, 2/3 */
  double h = 0.5 * x, h2 = h * h;
  double hm13 = pow(h, -1.0 / 3.0), hp13 = pow(h, 1.0 / 3.0);
  double hm23 = hm13 * hm13, hp23 = hp13 * hp13;
  /* I_{-1/3} = h^{-1/3}[1/G(2/3) + h^2/G(5/3)], I_{1/3} = h^{1/3}[1/G(4/3) + h^2/G(7/3)] */
  double k13 = c * (hm13 * (1.0 / g23 + h2 / g53) - hp13 * (1.0 / g43 + h2 / g73));
  double k23 = c * (hm23 * (1.0 / g13 + h2 / g43) - hp23 * (1.0 / g53 + h2 / g83));
  /* int_0^x (t/2)^p dt = 2 h^{p+1}/(p+1) */
  double ik = c * (2.0 * pow(h, 2.0 / 3.0) / (2.0 / 3.0) / g23 + 2.0 * pow(h, 8.0 / 3.0) / (8.0 / 3.0) / g53
                   - 2.0 * pow(h, 4.0 / 3.0) / (4.0 / 3.0) / g43 - 2.0 * pow(h, 10.0 / 3.0) / (10.0 / 3.0) / g73);
  double ex = exp(x);
  out[0] = ex * k13; out[1] = ex * k23; out[2] = ex * (OR_PI / sqrt(3.0) - ik);
}

void or_ktable(const or_ctx *c, double x, double out[3]) {
  if (x < 1e-3) { or_k_small(x, out); return; }
  if (x > 1e5) { double v = sqrt(OR_PI / (2.0 * x)); out[0] = out[1] = out[2] = v; return; }
  const double h = (K_HI - K_LO) / (NK - 1);
  double X = (log(x) - K_LO) / h;
  int i = (int)floor(X);
  if (i < 0) i = 0;
  if (i > NK - 2) i = NK - 2;
  double f = X - i;
  double f2 = f * f, f3 = f2 * f;
  double h00 = 2 * f3 - 3 * f2 + 1, h10 = f3 - 2 * f2 + f, h01 = -2 * f3 + 3 * f2, h11 = f3 - f2;
  for (int j = 0; j < 3; ++j)
    out[j] = h00 * c->kv[j][i] + h10 * h * c->kd[j][i] + h01 * c->kv[j][i + 1] + h11 * h * c->kd[j][i + 1];
}

/* 4-point Lagrange interpolation on a uniform grid, X in grid units */
static double or_lagrange4(const double *y, int n, double X) {
  if (X < 0) X = 0;
  if (X > n - 1) X = n - 1;
  int i = (int)floor(X);
  if (i < 1) i = 1;
  if (i > n - 3) i = n - 3;
  double f = X - i;
  double wm = -f * (f - 1) * (f - 2) / 6.0;
  double w0 = (f + 1) * (f - 1) * (f - 2) / 2.0;
  double w1 = -(f + 1) * f * (f - 2) / 2.0;
  double w2 = (f + 1) * f * (f - 1) / 6.0;
  return wm * y[i - 1] + w0 * y[i] + w1 * y[i + 1] + w2 * y[i + 2];
}

/* cubic Hermite along t for one row, T in grid units, h grid spacing */
static double or_hermite_row(const double *y, const double *d, int n, double T, double h) {
  if (T < 0) T = 0;
  if (T > n - 1) T = n - 1;
  int i = (int)floor(T);
  if (i < 0) i = 0;
  if (i > n - 2) i = n - 2;
  double f = T - i, f2 = f * f, f3 = f2 * f;
  return (2 * f3 - 3 * f2 + 1) * y[i] + (f3 - 2 * f2 + f) * h * d[i] + (-2 * f3 + 3 * f2) * y[i + 1] +
         (f3 - f2) * h * d[i + 1];
}

/* 2-D lookup: 4-point Lagrange across rows (ln chi), Hermite along t */
static double or_table2d(const double *Y, const double *D, int nx, int nt, double X, double T, double ht) {
  if (X < 0) X = 0;
  if (X > nx - 1) X = nx - 1;
  int i = (int)floor(X);
  if (i < 1) i = 1;
  if (i > nx - 3) i = nx - 3;
  double f = X - i;
  double w[4] = {-f * (f - 1) * (f - 2) / 6.0, (f + 1) * (f - 1) * (f - 2) / 2.0,
                 -(f + 1) * f * (f - 2) / 2.0, (f + 1) * f * (f - 1) / 6.0};
  double acc = 0;
  for (int k = 0; k < 4; ++k) {
    int row = i - 1 + k;
    acc += w[k] * or_hermite_row(Y + (size_t)row * nt, D + (size_t)row * nt, nt, T, ht);
  }
  return acc;
}

/* ---- Gauss-Legendre nodes/weights on [-1,1] (Newton on Legendre P_n) -------- */
static void or_gauleg(int n, double *x, double *w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), z1, pp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      z1 = z;
      z = z1 - p1 / pp;
      if (fabs(z - z1) < 1e-16) break;
    }
    x[i] = -z; x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}
static double GL8X[8], GL8W[8];
static double GL8B[8];  /* barycentric weights of the GL8 nodes */

static void or_gl8_bary(void) {
  or_gauleg(8, GL8X, GL8W);
  for (int j = 0; j < 8; ++j) {
    double p = 1.0;
    for (int k = 0; k < 8; ++k)
      if (k != j) p *= (GL8X[j] - GL8X[k]);
    GL8B[j] = 1.0 / p;
  }
}

/* value at xi in [-1,1] of the polynomial through (GL8X, fv) */
static double or_bary(const double fv[8], double xi) {
  double num = 0, den = 0;
  for (int j = 0; j < 8; ++j) {
    double d = xi - GL8X[j];
    if (d == 0.0) return fv[j];
    double t = GL8B[j] / d;
    num += t * fv[j]; den += t;
  }
  return num / den;
}

/* A panel's density is represented through the logarithms of its node values (the
 * density falls by many e-folds across a panel in the tails; its logarithm is smooth). */
static void or_logs(const double *f8, double lf[8]) {
  for (int k = 0; k < 8; ++k) lf[k] = f8[k] > 0.0 ? log(f8[k]) : -745.0;
}
static double or_dens(const double lf[8], double xi) { return exp(or_bary(lf, xi)); }

/* integral over [-1, xe] of exp(log-polynomial), by GL8 on the sub-interval */
static double or_dens_int(const double lf[8], double xe) {
  double half = 0.5 * (xe + 1.0), mid = 0.5 * (xe - 1.0), s = 0;
  for (int k = 0; k < 8; ++k) s += GL8W[k] * or_dens(lf, mid + half * GL8X[k]);
  return s * half;
}

/* Invert a panel-wise cumulative integral.  Panels p = 0..np-1 on [v0 + p H, v0+(p+1)H],
 * node values fv[p*8+k].  cum[p] = integral below panel p's left edge (cum[0] = tail),
 * target measured from below.  Returns v; *fout = density at v. */
static double or_invert_lower(const double *fv, const double *cum, int np, double v0, double H, double target,
                              double *fout) {
  if (target <= cum[0]) { /* analytic lower tail, integral ~ c e^{v/3}: F(v) = F(v0) e^{(v-v0)/3} */
    *fout = target / 3.0;  /* dF/dv = F/3 there */
    return v0 + 3.0 * log(target / cum[0]);
  }
  int lo = 0, hi = np;  /* find p with cum[p] <= target < cum[p+1] */
  while (hi - lo > 1) {
    int m = (lo + hi) / 2;
    if (cum[m] <= target) lo = m; else hi = m;
  }
  int p = lo;
  double lf[8];
  or_logs(fv + (size_t)p * 8, lf);
  double need = (target - cum[p]) / (0.5 * H);
  double total = (cum[p + 1] - cum[p]) / (0.5 * H);
  double a = -1.0, b = 1.0, xi = -1.0 + 2.0 * need / total;
  if (!(xi > a && xi < b)) xi = 0.0;
  for (int it = 0; it < 80; ++it) {
    double g = or_dens_int(lf, xi) - need;
    double fx = or_dens(lf, xi);
    if (g > 0) b = xi; else a = xi;
    double nx = (fx > 0) ? xi - g / fx : 0.5 * (a + b);
    if (!(nx > a && nx < b)) nx = 0.5 * (a + b);
    if (fabs(nx - xi) < 1e-15) { xi = nx; break; }
    xi = nx;
  }
  *fout = or_dens(lf, xi);
  return v0 + (p + 0.5 * (xi + 1.0)) * H;
}

/* same, measuring the target from above: cumu[p] = integral above panel p's left edge */
static double or_invert_upper(const double *fv, const double *cumu, int np, double v0, double H, double target,
                              double *fout) {
  int lo = 0, hi = np;  /* find p with cumu[p+1] <= target < cumu[p] */
  while (hi - lo > 1) {
    int m = (lo + hi) / 2;
    if (cumu[m] > target) lo = m; else hi = m;
  }
  int p = lo;
  double lf[8];
  or_logs(fv + (size_t)p * 8, lf);
  double above = (target - cumu[p + 1]) / (0.5 * H);   /* mass to leave above v in this panel */
  double a = -1.0, b = 1.0, xi = 0.0;
  /* integral from xi to +1 decreases with xi; solve it = above */
  for (int it = 0; it < 80; ++it) {
    double half = 0.5 * (1.0 - xi), mid = 0.5 * (1.0 + xi), s = 0;
    for (int k = 0; k < 8; ++k) s += GL8W[k] * or_dens(lf, mid + half * GL8X[k]);
    double g = above - s * half;   /* increases with xi */
    double fx = or_dens(lf, xi);
    if (g > 0) b = xi; else a = xi;
    double nx = (fx > 0) ? xi - g / fx : 0.5 * (a + b);
    if (!(nx > a && nx < b)) nx = 0.5 * (a + b);
    if (fabs(nx - xi) < 1e-15) { xi = nx; break; }
    xi = nx;
  }
  *fout = or_dens(lf, xi);
  return v0 + (p + 0.5 * (xi + 1.0)) * H;
}

/* ======================================================================= *
 *  NCS rate tables (Sec. III C).  Initial-spin-resolved, final-spin-summed *
 *  rate Eq. Wspin2 with W_R of Eq. F0's legend.  Reading: W_R carries 1/gamma *
 *  (the legend omits it; without it the chi<<1 power is not the classical *
 *  one).  Integrated over u:  W(chi, S) = alpha/(sqrt3 pi xi_L gamma)     *
 *  [A(chi) - (S.zeta) B(chi)],  zeta = n x a,                             *
 *   A = int du [(2+2u+u^2)K23(u') - (1+u)IntK13(u')]/(1+u)^3,             *
 *   B = int du u K13(u')/(1+u)^3,   u' = 2u/(3chi).                       *
 *  Quadrature: u = 1.5 chi u', v = ln u' on 8-point Gauss panels.          *
 * ======================================================================= */
#define NCS_V0 (-120.0)
#define NCS_V1 (7.0)
#define NCS_H 0.25
#define NCS_NP 508

static void or_ncs_density(double chi, double up, const double ks[3], double *fa, double *fb) {
  double u = 1.5 * chi * up;
  double em = exp(-up);
  double k13 = ks[0] * em, k23 = ks[1] * em, ik = ks[2] * em;
  double q = 1.0 + u, q3 = q * q * q;
  double jac = 1.5 * chi * up;   /* du/dv */
  *fa = jac * ((2.0 + 2.0 * u + u * u) * k23 - q * ik) / q3;
  *fb = jac * (u * k13) / q3;
}

static void or_build_ncs(or_ctx *c) {
  const int nn = NCS_NP * 8;
  double *up = (double *)malloc(sizeof(double) * nn);
  double *ks = (double *)malloc(sizeof(double) * nn * 3);
  for (int p = 0; p < NCS_NP; ++p)
    for (int k = 0; k < 8; ++k) {
      double v = NCS_V0 + (p + 0.5 * (GL8X[k] + 1.0)) * NCS_H;
      up[p * 8 + k] = exp(v);
      or_besselk_scaled(up[p * 8 + k], ks + (size_t)(p * 8 + k) * 3);
    }
  double ks0[3], up0 = exp(NCS_V0);
  or_besselk_scaled(up0, ks0);

  /* rate table */
  const double hr = (R_HI - R_LO) / (NR - 1);
  for (int i = 0; i < NR; ++i) {
    double chi = exp(R_LO + i * hr);
    double fa0, fb0;
    or_ncs_density(chi, up0, ks0, &fa0, &fb0);
    double A = 3.0 * fa0, B = 0.6 * fb0;  /* tails below v0: ~e^{v/3} and ~e^{5v/3} */
    for (int p = 0; p < NCS_NP; ++p) {
      double sa = 0, sb = 0;
      for (int k = 0; k < 8; ++k) {
        double fa, fb;
        or_ncs_density(chi, up[p * 8 + k], ks + (size_t)(p * 8 + k) * 3, &fa, &fb);
        sa += GL8W[k] * fa; sb += GL8W[k] * fb;
      }
      A += sa * NCS_H * 0.5; B += sb * NCS_H * 0.5;
    }
    c->ra[i] = A / chi; c->rb[i] = B / chi;
    /* radiative pusher functions on the same nodes (Sec. III A, B):
     *   q(chi) = I_QED / I_C, the quantum radiated power over the classical one,
     *     I_QED = alpha/(sqrt3 pi xi_L) int du u/(1+u) [(2+2u+u^2)K23 - (1+u)IntK13]/(1+u)^3
     *     (photon energy omega = gamma u/(1+u) times the rate of Eq. Wspin2, spin-averaged),
     *     I_C = (2/3) alpha chi^2 / xi_L  =>  q = sqrt3/(2 pi chi^2) int du (...);
     *   psi1 = int du u'' K23(u'), psi3 = int du u'' K13(u'),
     *   psi2 = int du u'' IntK13(u') - psi1,  u'' = u^2/(1+u)^3  (Eq. spin1's legend).
     * Below v0 every density is O(u'^{4/3}) or smaller: no tail term. */
    double I[4] = {0, 0, 0, 0};
    for (int p = 0; p < NCS_NP; ++p) {
      double s4[4] = {0, 0, 0, 0};
      for (int k = 0; k < 8; ++k) {
        const double *kk = ks + (size_t)(p * 8 + k) * 3;
        double upk = up[p * 8 + k], u = 1.5 * chi * upk, em = exp(-upk), qq = 1.0 + u;
        double jac = 1.5 * chi * upk, upp = u * u / (qq * qq * qq);
        double fa, fb;
        or_ncs_density(chi, upk, kk, &fa, &fb);
        s4[0] += GL8W[k] * fa * u / qq;
        s4[1] += GL8W[k] * jac * upp * kk[1] * em;
        s4[2] += GL8W[k] * jac * upp * kk[2] * em;
        s4[3] += GL8W[k] * jac * upp * kk[0] * em;
      }
      for (int j = 0; j < 4; ++j) I[j] += s4[j] * NCS_H * 0.5;
    }
    double chi3 = chi * chi * chi;
    c->rr[0][i] = sqrt(3.0) / (2.0 * OR_PI * chi * chi) * I[0];
    c->rr[1][i] = I[1] / chi3;
    c->rr[2][i] = (I[2] - I[1]) / chi3;
    c->rr[3][i] = I[3] / chi3;
  }

  /* inverse CDF tables: component 0 = spin projection s=+1 (a-b), 1 = s=-1 (a+b) */
  double *fv = (double *)malloc(sizeof(double) * nn);
  double *cum = (double *)malloc(sizeof(double) * (NCS_NP + 1));
  double *cumu = (double *)malloc(sizeof(double) * (NCS_NP + 1));
  double *pint = (double *)malloc(sizeof(double) * NCS_NP);
  const double hx = (R_HI - R_LO) / (NCX - 1);
  const double ht = (CT_HI - CT_LO) / (NCT - 1);
  for (int comp = 0; comp < 2; ++comp) {
    double sg = comp == 0 ? -1.0 : 1.0;
    for (int i = 0; i < NCX; ++i) {
      double chi = exp(R_LO + i * hx);
      for (int j = 0; j < nn; ++j) {
        double fa, fb;
        or_ncs_density(chi, up[j], ks + (size_t)j * 3, &fa, &fb);
        fv[j] = fa + sg * fb;
      }
      double fa0, fb0;
      or_ncs_density(chi, up0, ks0, &fa0, &fb0);
      cum[0] = 3.0 * (fa0 + sg * fb0);
      for (int p = 0; p < NCS_NP; ++p) {
        double s = 0;
        for (int k = 0; k < 8; ++k) s += GL8W[k] * fv[p * 8 + k];
        pint[p] = s * NCS_H * 0.5;
        cum[p + 1] = cum[p] + pint[p];
      }
      /* mass above each panel edge, summed from the top (no differences of large sums) */
      cumu[NCS_NP] = 0;
      for (int p = NCS_NP - 1; p >= 0; --p) cumu[p] = cumu[p + 1] + pint[p];
      double tot = cum[NCS_NP];
      double lnscale = log(1.5 * chi);
      for (int j = 0; j < NCT; ++j) {
        double t = CT_LO + j * ht;
        double v, fvv;
        double lq = 1.0 / (1.0 + exp(-t)), lp = 1.0 / (1.0 + exp(t));   /* l, 1-l */
        if (t <= 0) v = or_invert_lower(fv, cum, NCS_NP, NCS_V0, NCS_H, lq * tot, &fvv);
        else v = or_invert_upper(fv, cumu, NCS_NP, NCS_V0, NCS_H, lp * tot, &fvv);
        c->cy[comp][i][j] = v + lnscale;
        c->cd[comp][i][j] = lq * lp * tot / fvv;
      }
    }
  }
  free(fv); free(cum); free(cumu); free(pint); free(up); free(ks);
}

/* ======================================================================= *
 *  NBW tables (Sec. III D).  Spin-summed rate per d(epsilon_+) from        *
 *  Eq. BW summed over S+ and S- (Eqs. G0, G3): W0 {IntK13 + (e-^2+e+^2)/   *
 *  (e-e+) K23 - xi3 K23}.  Readings: Eq. BWprob's 2W0 and Eq. BW_pos's W0 *
 *  are twice the sum of Eq. BW with the W0/2 in G0..G3; rho carries chi_g *
 *  (Eq. rho as printed omits it); times 1/xi_L for normalised time.       *
 *  Per d delta: alpha/(sqrt3 pi xi_L omega)[t0(delta) - xi3 t3(delta)],   *
 *  T0,T3 = int_0^1 d delta; stored scaled by exp(8/(3chi_g)).             *
 *  Variable: delta = 1/(1+e^{-s}), s<=0 (the density is symmetric).       *
 * ======================================================================= */
#define NBW_S0 (-16.0)
#define NBW_H (1.0 / 16.0)
#define NBW_NP 256

static void or_nbw_density(double chig, double s, double *ft0, double *ft3, double *delta) {
  double d = 1.0 / (1.0 + exp(-s));
  double om = 1.0 / (1.0 + exp(s));
  double dd = d * om;
  double rho = 2.0 / (3.0 * chig * dd);
  double ex = (2.0 / (3.0 * chig)) * (1.0 - 2.0 * d) * (1.0 - 2.0 * d) / dd;  /* rho - 8/(3chig) */
  *delta = d;
  if (ex > 740.0) { *ft0 = 0; *ft3 = 0; return; }
  double ks[3];
  or_besselk_scaled(rho, ks);
  double e = exp(-ex);
  double k23 = ks[1] * e, ik = ks[2] * e;
  *ft0 = dd * (ik + (d / om + om / d) * k23);
  *ft3 = dd * k23;
}

static void or_build_nbw(or_ctx *c) {
  const int nn = NBW_NP * 8;
  double *f0 = (double *)malloc(sizeof(double) * nn), *f3 = (double *)malloc(sizeof(double) * nn);
  double *fv = (double *)malloc(sizeof(double) * nn);
  double *cum = (double *)malloc(sizeof(double) * (NBW_NP + 1));
  const double hx = (B_HI - B_LO) / (NBX - 1);
  const double ht = (BT_HI - BT_LO) / (NBT - 1);
  for (int i = 0; i < NBX; ++i) {
    double chig = exp(B_LO + i * hx);
    double T0 = 0, T3 = 0;
    for (int p = 0; p < NBW_NP; ++p)
      for (int k = 0; k < 8; ++k) {
        double s = NBW_S0 + (p + 0.5 * (GL8X[k] + 1.0)) * NBW_H, dl;
        or_nbw_density(chig, s, &f0[p * 8 + k], &f3[p * 8 + k], &dl);
        T0 += GL8W[k] * f0[p * 8 + k] * NBW_H * 0.5;
        T3 += GL8W[k] * f3[p * 8 + k] * NBW_H * 0.5;
      }
    c->t0s[i] = 2.0 * T0; c->t3s[i] = 2.0 * T3;
    for (int comp = 0; comp < 2; ++comp) {
      double sg = comp == 0 ? -1.0 : 1.0;   /* 0: xi3'=+1 -> t0 - t3 */
      for (int j = 0; j < nn; ++j) fv[j] = f0[j] + sg * f3[j];
      cum[0] = 0;
      for (int p = 0; p < NBW_NP; ++p) {
        double s = 0;
        for (int k = 0; k < 8; ++k) s += GL8W[k] * fv[p * 8 + k];
        cum[p + 1] = cum[p] + s * NBW_H * 0.5;
      }
      double half = cum[NBW_NP];
      for (int j = 0; j < NBT; ++j) {
        double t = BT_LO + j * ht;
        double lam = exp(t);
        double s, fs;
        if (j == NBT - 1) {
          double a0, a3, dd;
          s = 0.0;
          or_nbw_density(chig, s, &a0, &a3, &dd);
          fs = a0 + sg * a3;
        } else {
          s = or_invert_lower(fv, cum, NBW_NP, NBW_S0, NBW_H, lam * half, &fs);
        }
        double dl = 1.0 / (1.0 + exp(-s));
        c->by[comp][i][j] = log(dl);
        c->bd[comp][i][j] = (1.0 - dl) * lam * half / fs;
      }
    }
  }
  free(f0); free(f3); free(fv); free(cum);
}

/* ======================================================================= *
 *  Vacuum birefringence (Sec. III F, Eq. eqnn and the M definition).      *
 *  Scorer Gi'(y) for y > 0: rotating the contour of Gi(y) = (1/pi) int_0^  *
 *  inf sin(t^3/3 + y t) dt by pi/6 gives                                   *
 *   pi Gi'(y) = int_0^inf s exp(-s^3/3 - y s/2) cos(pi/3 + sqrt3 y s/2) ds. *
 *  Trapezoid in w = ln s.                                                  *
 *  M(chi_g) = -(45/4) int_0^1 dv (1-v^2){(1+v^2/3)/2 ; 1-v^2/3}           *
 *             pi x^{4/3} Gi'(x^{2/3}),  x = 4/((1-v^2) chi_g).             *
 * ======================================================================= */
double or_scorer_gi_prime(double y) {
  double smax = 5.5;
  if (100.0 / y < smax) smax = 100.0 / y;
  double wmax = log(1.2 * smax);
  double wmin = log(1e-9) - (y > 1.0 ? log(y) : 0.0);
  const double h = 0.04;
  int n = (int)ceil((wmax - wmin) / h);
  double s3 = sqrt(3.0), acc = 0;
  for (int k = 0; k <= n; ++k) {
    double w = wmin + k * h, s = exp(w);
    double term = s * s * exp(-s * s * s / 3.0 - 0.5 * y * s) * cos(OR_PI / 3.0 + 0.5 * s3 * y * s);
    acc += (k == 0 || k == n) ? 0.5 * term : term;
  }
  return acc * h / OR_PI;
}

/* The upsilon integral: the integrand changes shape in a layer of width ~1/chi_g next to
 * upsilon = 1 (where x grows from O(1) to infinity), so the interval is split into [0, 1/2]
 * and panels [1 - 2^-k, 1 - 2^-(k+1)], k = 1..30, each with 8-point Gauss; the remainder
 * next to 1 contributes below 1e-18. */
static void or_vb_exact(double chig, double out[2]) {
  double mp = 0, mq = 0;
  for (int k = 0; k <= 30; ++k) {
    double a = (k == 0) ? 0.0 : 1.0 - ldexp(1.0, -k);
    double b = 1.0 - ldexp(1.0, -(k + 1));
    double hm = 0.5 * (b - a), c = 0.5 * (b + a);
    for (int j = 0; j < 8; ++j) {
      double v = c + hm * GL8X[j], wv = hm * GL8W[j];
      double omv = 1.0 - v * v;
      double x = 4.0 / (omv * chig);
      double y = pow(x, 2.0 / 3.0);
      double g = OR_PI * y * y * or_scorer_gi_prime(y);   /* = pi x^{4/3} Gi'(x^{2/3}) */
      mp += wv * omv * 0.5 * (1.0 + v * v / 3.0) * g;
      mq += wv * omv * (1.0 - v * v / 3.0) * g;
    }
  }
  out[0] = -11.25 * mp; out[1] = -11.25 * mq;
}

/* ======================================================================= */
or_ctx *or_ctx_create(void) {
  or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
  if (!c) return NULL;
  or_gl8_bary();
  const double h = (K_HI - K_LO) / (NK - 1);
  for (int i = 0; i < NK; ++i) {
    double x = exp(K_LO + i * h), k[3];
    or_besselk_scaled(x, k);
    for (int j = 0; j < 3; ++j) c->kv[j][i] = k[j];
    /* exact derivatives d/d ln x of the scaled functions (DLMF 10.29.2) */
    c->kd[0][i] = x * (k[0] - k[1]) - k[0] / 3.0;
    c->kd[1][i] = x * (k[1] - k[0]) - 2.0 * k[1] / 3.0;
    c->kd[2][i] = x * (k[2] - k[0]);
  }
  or_build_ncs(c);
  or_build_nbw(c);
  const double hv = (V_HI - V_LO) / (NV - 1);
  for (int i = 0; i < NV; ++i) {
    double m[2];
    or_vb_exact(exp(V_LO + i * hv), m);
    c->mpar[i] = m[0]; c->mperp[i] = m[1];
  }
  c->near_tol = 1e-6;
  c->threads = 1;
  c->logcap = 1 << 20;
  c->log_id = (uint64_t *)malloc(sizeof(uint64_t) * c->logcap);
  c->log_step = (uint32_t *)malloc(sizeof(uint32_t) * c->logcap);
  c->log_kind = (uint32_t *)malloc(sizeof(uint32_t) * c->logcap);
  c->log_margin = (double *)malloc(sizeof(double) * c->logcap);
  return c;
}

void or_ctx_destroy(or_ctx *c) {
  if (!c) return;
  free(c->log_id); free(c->log_step); free(c->log_kind); free(c->log_margin);
  free(c->p_be); free(c->p_bp); free(c->p_bg); free(c->p_dec);   /* an uncommitted step */
  free(c);
}
void or_set_next_id(or_ctx *c, uint64_t id) { c->next_id = id; c->nlog = 0; }
uint64_t or_get_next_id(const or_ctx *c) { return c->next_id; }
void or_set_near_tol(or_ctx *c, double tol) { c->near_tol = tol; }
int or_set_threads(or_ctx *c, int n) {
#ifdef _OPENMP
  c->threads = n < 1 ? 1 : n;
#else
  (void)n;
  c->threads = 1;
#endif
  return c->threads;
}
uint64_t or_near_log(or_ctx *c, uint64_t *ids, uint32_t *steps, uint32_t *kinds, double *margins, uint64_t cap) {
  uint64_t n = c->nlog < c->logcap ? c->nlog : c->logcap;
  n = n < cap ? n : cap;
  for (uint64_t i = 0; i < n; ++i) {
    ids[i] = c->log_id[i]; steps[i] = c->log_step[i]; kinds[i] = c->log_kind[i]; margins[i] = c->log_margin[i];
  }
  return c->nlog;
}

const double *or_table(const or_ctx *c, int which, uint64_t *len) {
  switch (which) {
    case 0: *len = 6 * NK; return &c->kv[0][0];
    case 1: *len = 2 * NR; return c->ra;
    case 2: *len = 4 * NCX * NCT; return &c->cy[0][0][0];
    case 3: *len = 2 * NBX; return c->t0s;
    case 4: *len = 4 * NBX * NBT; return &c->by[0][0][0];
    case 5: *len = 2 * NV; return c->mpar;
    case 6: *len = 4 * NR; return &c->rr[0][0];
    case 7: *len = 2 * NMG * NMS; return &c->mb[0][0];   /* mb then mp (contiguous) */
  }
  *len = 0;
  return NULL;
}

void or_ncs_rates(const or_ctx *c, double chi, double out[2]) {
  double X = (log(chi) - R_LO) / ((R_HI - R_LO) / (NR - 1));
  out[0] = chi * or_lagrange4(c->ra, NR, X);
  out[1] = chi * or_lagrange4(c->rb, NR, X);
}
double or_ncs_invcdf(const or_ctx *c, int comp, double chi, double t) {
  double X = (log(chi) - R_LO) / ((R_HI - R_LO) / (NCX - 1));
  double ht = (CT_HI - CT_LO) / (NCT - 1);
  return or_table2d(&c->cy[comp][0][0], &c->cd[comp][0][0], NCX, NCT, X, (t - CT_LO) / ht, ht);
}
void or_nbw_rates(const or_ctx *c, double chig, double out[2]) {
  double X = (log(chig) - B_LO) / ((B_HI - B_LO) / (NBX - 1));
  double damp = exp(-8.0 / (3.0 * chig));
  out[0] = damp * or_lagrange4(c->t0s, NBX, X);
  out[1] = damp * or_lagrange4(c->t3s, NBX, X);
}
double or_nbw_invcdf(const or_ctx *c, int comp, double chig, double t) {
  double X = (log(chig) - B_LO) / ((B_HI - B_LO) / (NBX - 1));
  double ht = (BT_HI - BT_LO) / (NBT - 1);
  return or_table2d(&c->by[comp][0][0], &c->bd[comp][0][0], NBX, NBT, X, (t - BT_LO) / ht, ht);
}
/* q and psi1..3 at chi from the tables (4-point Lagrange in ln chi).  Below chi_min:
 * q = 1 (its classical limit) and psi_i = chi^3 times the first node's psi_i/chi^3
 * (the psi's go as chi^3 for chi -> 0); above chi_max the caller clamps chi. */
void or_rr_funcs(const or_ctx *c, double chi, double out[4]) {
  double X = (log(chi) - R_LO) / ((R_HI - R_LO) / (NR - 1));
  double chi3 = chi * chi * chi;
  out[0] = chi < OR_CHI_MIN ? 1.0 : or_lagrange4(c->rr[0], NR, X);
  for (int j = 1; j < 4; ++j) out[j] = chi3 * or_lagrange4(c->rr[j], NR, X);
}

void or_vb_m(const or_ctx *c, double chig, double out[2]) {
  if (chig < OR_VB_MIN) { out[0] = 4.0; out[1] = 7.0; return; }
  double X = (log(chig) - V_LO) / ((V_HI - V_LO) / (NV - 1));
  out[0] = or_lagrange4(c->mpar, NV, X);
  out[1] = or_lagrange4(c->mperp, NV, X);
}

/* ======================================================================= *
 *  Vector helpers                                                          *
 * ======================================================================= */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double o[3]) {
  double x = a[1] * b[2] - a[2] * b[1], y = a[2] * b[0] - a[0] * b[2], z = a[0] * b[1] - a[1] * b[0];
  o[0] = x; o[1] = y; o[2] = z;
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* canonical transverse frame of a direction n (basis-angle reference):
 * e1 = unit(y x n), fallback unit(n x x) when n is within 1e-10 of +-y; e2 = n x e1 */
static void or_frame(const double n[3], double e1[3], double e2[3]) {
  double a = n[2], b = 0.0, cc = -n[0];
  double m2 = a * a + cc * cc;
  if (m2 < 1e-20) { a = 0.0; b = n[2]; cc = -n[1]; m2 = b * b + cc * cc; }
  double inv = 1.0 / sqrt(m2);
  e1[0] = a * inv; e1[1] = b * inv; e1[2] = cc * inv;
  cross3(n, e1, e2);
}

/* ======================================================================= *
 *  External fields (Sec. II D force deposition, E field models)           *
 * ======================================================================= */
static double or_env(const or_fields *f, double phi) {
  double s = (phi - f->phi0) / f->len;
  if (s < 0.0 || s > 1.0) return 0.0;
  double sn = sin(OR_PI * s);
  return sn * sn;
}

/* TSC weights of Sec. II E (reading: the j+-1 weights are (1/2)(1/2 -+ delta)^2) */
static void or_tsc(double d, double w[3]) {
  w[0] = 0.5 * (0.5 - d) * (0.5 - d);
  w[1] = 0.75 - d * d;
  w[2] = 0.5 * (0.5 + d) * (0.5 + d);
}

/* node index on a grid axis of n nodes: wrapped (periodic) or -1 when outside */
static int or_node(int i, int n, int periodic) {
  if (periodic) { i %= n; return i < 0 ? i + n : i; }
  return (i < 0 || i >= n) ? -1 : i;
}

static double or_gather(const float *g, int nx, int ny, int periodic, double xs, double ys, int hx, int hy) {
  /* hx, hy: 1 if the component sits on the half grid along that axis */
  double X = hx ? xs - 0.5 : xs, Y = hy ? ys - 0.5 : ys;
  int ig = (int)floor(X + 0.5), jg = (int)floor(Y + 0.5);
  double wx[3], wy[3];
  or_tsc(X - ig, wx);
  or_tsc(Y - jg, wy);
  double acc = 0;
  for (int b = 0; b < 3; ++b) {
    int j = or_node(jg - 1 + b, ny, periodic);
    if (j < 0) continue;
    for (int a = 0; a < 3; ++a) {
      int i = or_node(ig - 1 + a, nx, periodic);
      if (i < 0) continue;
      acc += wx[a] * wy[b] * (double)g[(size_t)j * nx + i];
    }
  }
  return acc;
}

/* ======================================================================= *
 *  Esirkepov current deposition (Sec. II C, Esirkepov 2001) with the TSC  *
 *  shape of Sec. II E, 2D3V.  The particle moves from (X0, Y0) to (X1, Y1) *
 *  in cell units during dt (less than half a cell per axis, the CFL of    *
 *  the field solver).  Shapes S0, S1 on the 5 nodes around the old       *
 *  nearest node; DS = S1 - S0;                                            *
 *    Wx = DS_x (S0_y + DS_y/2), Wy = DS_y (S0_x + DS_x/2),                 *
 *    Wz = S0_x S0_y + DS_x S0_y/2 + S0_x DS_y/2 + DS_x DS_y/3;             *
 *  Jx(i+1/2,j) = -(q w/(dy dt)) sum_{i'<=i} Wx(i',j),                      *
 *  Jy(i,j+1/2) = -(q w/(dx dt)) sum_{j'<=j} Wy(i,j'),                      *
 *  Jz(i,j) = q w vz Wz(i,j)/(dx dy),                                       *
 *  which makes (rho^{n+1} - rho^n)/dt + div J = 0 on the grid exactly.     *
 * ======================================================================= */
static void or_deposit(const or_fields *f, double qw, const double xo[3], const double xn[3], double vz,
                       double dt) {
  double X0 = (xo[0] - f->x0) / f->dx, Y0 = (xo[1] - f->y0) / f->dy;
  double X1 = (xn[0] - f->x0) / f->dx, Y1 = (xn[1] - f->y0) / f->dy;
  int i0 = (int)floor(X0 + 0.5), j0 = (int)floor(Y0 + 0.5);
  int i1 = (int)floor(X1 + 0.5), j1 = (int)floor(Y1 + 0.5);
  double S0x[5] = {0}, S1x[5] = {0}, S0y[5] = {0}, S1y[5] = {0}, w[3];
  int di = i1 - i0, dj = j1 - j0;
  if (di < -1 || di > 1 || dj < -1 || dj > 1) return;   /* beyond the solver's CFL: not deposited */
  or_tsc(X0 - i0, w);
  for (int k = 0; k < 3; ++k) S0x[1 + k] = w[k];
  or_tsc(X1 - i1, w);
  for (int k = 0; k < 3; ++k) S1x[1 + di + k] = w[k];
  or_tsc(Y0 - j0, w);
  for (int k = 0; k < 3; ++k) S0y[1 + k] = w[k];
  or_tsc(Y1 - j1, w);
  for (int k = 0; k < 3; ++k) S1y[1 + dj + k] = w[k];
  const double cx = -qw / (f->dy * dt), cy = -qw / (f->dx * dt), cz = qw * vz / (f->dx * f->dy);
  for (int b = 0; b < 5; ++b) {
    int j = or_node(j0 - 2 + b, f->ny, f->periodic);
    double acc = 0.0;
    for (int a = 0; a < 5; ++a) {
      double dsx = S1x[a] - S0x[a], dsy = S1y[b] - S0y[b];
      double Wx = dsx * (S0y[b] + 0.5 * dsy);
      double Wz = S0x[a] * S0y[b] + 0.5 * dsx * S0y[b] + 0.5 * S0x[a] * dsy + dsx * dsy / 3.0;
      acc += Wx;
      int i = or_node(i0 - 2 + a, f->nx, f->periodic);
      if (i < 0 || j < 0) continue;
      if (a < 4) f->gJx[(size_t)j * f->nx + i] += cx * acc;
      f->gJz[(size_t)j * f->nx + i] += cz * Wz;
    }
  }
  for (int a = 0; a < 5; ++a) {
    int i = or_node(i0 - 2 + a, f->nx, f->periodic);
    double acc = 0.0;
    for (int b = 0; b < 5; ++b) {
      double dsx = S1x[a] - S0x[a], dsy = S1y[b] - S0y[b];
      acc += dsy * (S0x[a] + 0.5 * dsx);
      int j = or_node(j0 - 2 + b, f->ny, f->periodic);
      if (i < 0 || j < 0 || b == 4) continue;
      f->gJy[(size_t)j * f->nx + i] += cy * acc;
    }
  }
}

/* ======================================================================= *
 *  Yee field solver (Sec. II B), 2D (z squeezed), the curl equations only *
 *  (Gauss's law is kept by the charge-conserving deposition).  Neighbours *
 *  outside the grid are zero, or wrap when periodic.                       *
 * ======================================================================= */
static double or_at(const double *a, const or_grid *g, int i, int j) {
  i = or_node(i, g->nx, g->periodic);
  j = or_node(j, g->ny, g->periodic);
  return (i < 0 || j < 0) ? 0.0 : a[(size_t)j * g->nx + i];
}

void or_fdtd_b(const or_grid *g, double dt) {
  const int nx = g->nx, ny = g->ny;
  double *nbx = (double *)malloc(sizeof(double) * nx * ny), *nby = (double *)malloc(sizeof(double) * nx * ny);
  double *nbz = (double *)malloc(sizeof(double) * nx * ny);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = (size_t)j * nx + i;
      /* Bx(i,j+1/2): -dEz/dy;  By(i+1/2,j): +dEz/dx;  Bz(i+1/2,j+1/2): -(dEy/dx - dEx/dy) */
      nbx[k] = g->Bx[k] - dt * (or_at(g->Ez, g, i, j + 1) - or_at(g->Ez, g, i, j)) / g->dy;
      nby[k] = g->By[k] + dt * (or_at(g->Ez, g, i + 1, j) - or_at(g->Ez, g, i, j)) / g->dx;
      nbz[k] = g->Bz[k] - dt * ((or_at(g->Ey, g, i + 1, j) - or_at(g->Ey, g, i, j)) / g->dx -
                                (or_at(g->Ex, g, i, j + 1) - or_at(g->Ex, g, i, j)) / g->dy);
    }
  memcpy(g->Bx, nbx, sizeof(double) * nx * ny);
  memcpy(g->By, nby, sizeof(double) * nx * ny);
  memcpy(g->Bz, nbz, sizeof(double) * nx * ny);
  free(nbx); free(nby); free(nbz);
}

void or_fdtd_e(const or_grid *g, double dt) {
  const int nx = g->nx, ny = g->ny;
  double *nex = (double *)malloc(sizeof(double) * nx * ny), *ney = (double *)malloc(sizeof(double) * nx * ny);
  double *nez = (double *)malloc(sizeof(double) * nx * ny);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = (size_t)j * nx + i;
      /* Ex(i+1/2,j): dBz/dy - Jx;  Ey(i,j+1/2): -dBz/dx - Jy;  Ez(i,j): dBy/dx - dBx/dy - Jz */
      nex[k] = g->Ex[k] + dt * ((or_at(g->Bz, g, i, j) - or_at(g->Bz, g, i, j - 1)) / g->dy - g->Jx[k]);
      ney[k] = g->Ey[k] + dt * (-(or_at(g->Bz, g, i, j) - or_at(g->Bz, g, i - 1, j)) / g->dx - g->Jy[k]);
      nez[k] = g->Ez[k] + dt * ((or_at(g->By, g, i, j) - or_at(g->By, g, i - 1, j)) / g->dx -
                                (or_at(g->Bx, g, i, j) - or_at(g->Bx, g, i, j - 1)) / g->dy - g->Jz[k]);
    }
  memcpy(g->Ex, nex, sizeof(double) * nx * ny);
  memcpy(g->Ey, ney, sizeof(double) * nx * ny);
  memcpy(g->Ez, nez, sizeof(double) * nx * ny);
  free(nex); free(ney); free(nez);
}

void or_charge_tsc(const or_grid *g, double x0, double y0, const double *x, const double *y, const double *qw,
                   uint64_t n, double *rho) {
  for (uint64_t p = 0; p < n; ++p) {
    double X = (x[p] - x0) / g->dx, Y = (y[p] - y0) / g->dy;
    int ig = (int)floor(X + 0.5), jg = (int)floor(Y + 0.5);
    double wx[3], wy[3];
    or_tsc(X - ig, wx);
    or_tsc(Y - jg, wy);
    for (int b = 0; b < 3; ++b) {
      int j = or_node(jg - 1 + b, g->ny, g->periodic);
      if (j < 0) continue;
      for (int a = 0; a < 3; ++a) {
        int i = or_node(ig - 1 + a, g->nx, g->periodic);
        if (i < 0) continue;
        rho[(size_t)j * g->nx + i] += qw[p] * wx[a] * wy[b] / (g->dx * g->dy);
      }
    }
  }
}

void or_field(const or_fields *f, double x, double y, double z, double t, double E[3], double B[3]) {
  E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.0;
  if (f->kind == OR_FIELD_UNIFORM) {
    for (int k = 0; k < 3; ++k) { E[k] = f->E[k]; B[k] = f->B[k]; }
  } else if (f->kind == OR_FIELD_PLANE) {
    /* plane wave along -z, phase phi = t + z; B = k x E with k = -z */
    double phi = t + z;
    double g = f->a0 * or_env(f, phi);
    if (g == 0.0) return;
    E[0] = g * cos(phi);
    E[1] = f->circular ? g * sin(phi) : 0.0;
    B[0] = E[1]; B[1] = -E[0];
  } else if (f->kind == OR_FIELD_GAUSS) {
    /* first-order paraxial Gaussian along -z, focus at z = zf; longitudinal
       components neglected; B = k x E_perp */
    double phi = t + z;
    double g = f->a0 * or_env(f, phi);
    if (g == 0.0) return;
    double zeta = f->zf - z;                 /* distance travelled past focus */
    double zr = 0.5 * f->w0 * f->w0;
    double q = zeta / zr;
    double w2 = f->w0 * f->w0 * (1.0 + q * q);
    double r2 = x * x + y * y;
    double amp = g * (f->w0 / sqrt(w2)) * exp(-r2 / w2);
    double ph = phi - 0.5 * r2 * zeta / (zeta * zeta + zr * zr) + atan(q);
    E[0] = amp * cos(ph);
    E[1] = f->circular ? amp * sin(ph) : 0.0;
    B[0] = E[1]; B[1] = -E[0];
  } else if (f->kind == OR_FIELD_GRID2D) {
    /* 2D Yee staggering (z squeezed): Ex(i+1/2,j) Ey(i,j+1/2) Ez(i,j)
       Bx(i,j+1/2) By(i+1/2,j) Bz(i+1/2,j+1/2) */
    double xs = (x - f->x0) / f->dx, ys = (y - f->y0) / f->dy;
    E[0] = or_gather(f->gEx, f->nx, f->ny, f->periodic, xs, ys, 1, 0);
    E[1] = or_gather(f->gEy, f->nx, f->ny, f->periodic, xs, ys, 0, 1);
    E[2] = or_gather(f->gEz, f->nx, f->ny, f->periodic, xs, ys, 0, 0);
    B[0] = or_gather(f->gBx, f->nx, f->ny, f->periodic, xs, ys, 0, 1);
    B[1] = or_gather(f->gBy, f->nx, f->ny, f->periodic, xs, ys, 1, 0);
    B[2] = or_gather(f->gBz, f->nx, f->ny, f->periodic, xs, ys, 1, 1);
  }
}

/* ======================================================================= *
 *  NCS photon-polarisation- and spin-resolved functions F0..F3            *
 *  (Eqs. F0, F1, F2, F3 as printed; u' = 2u/(3chi); K's scaled by e^{u'}, *
 *  a common factor).  zeta = n x a.                                        *
 * ======================================================================= */
void or_ncs_F(const or_ctx *c, double u, double chi, const double n[3], const double a[3],
              const double Si[3], const double Sf[3], double F[4]) {
  double ks[3];
  or_ktable(c, 2.0 * u / (3.0 * chi), ks);
  double K13 = ks[0], K23 = ks[1], IK = ks[2];
  double z[3];
  cross3(n, a, z);
  double Sif = dot3(Si, Sf);
  double Siz = dot3(Si, z), Sfz = dot3(Sf, z);
  double Sin = dot3(Si, n), Sfn = dot3(Sf, n);
  double Sia = dot3(Si, a), Sfa = dot3(Sf, a);
  double fxs[3];
  cross3(Sf, Si, fxs);
  double u2 = u * u;
  F[0] = -(2 + u) * (2 + u) * (IK - 2 * K23) * (1 + Sif) + u2 * (1 - Sif) * (IK + 2 * K23) + 2 * u2 * Sif * IK -
         (4 * u + 2 * u2) * (Sfz + Siz) * K13 - 2 * u2 * (Sfz - Siz) * K13 - 4 * u2 * (IK - K23) * Sin * Sfn;
  F[1] = -2 * u2 * IK * (Sia * Sfz + Sfa * Siz) + 4 * u * (Sia * (1 + u) + Sfa) * K13 +
         2 * u * (2 + u) * dot3(n, fxs) * K23;
  F[2] = -(2 * u2 * (Sin * Sfz + Sfn * Siz) + 2 * u * (2 + u) * dot3(a, fxs)) * K13 -
         4 * u * (Sin + Sfn * (1 + u)) * IK + 4 * u * (2 + u) * (Sin + Sfn) * K23;
  F[3] = 4 * (1 + u + (1 + u + 0.5 * u2) * Sif - 0.5 * u2 * Sin * Sfn) * K23 + 2 * u2 * (Siz * Sfz - Sia * Sfa) * IK -
         4 * u * ((1 + u) * Siz + Sfz) * K13;
}

/* ======================================================================= *
 *  NBW polarisation/spin-resolved functions G0..G3 (Eqs. G0-G3 as printed, *
 *  reading: a, b in G1's last term are a+, b+; common W0/2 dropped; K's   *
 *  scaled by e^rho, a common factor).                                      *
 * ======================================================================= */
void or_nbw_G(const or_ctx *c, double delta, double omega, double chig, const double ap[3], const double bp[3],
              const double vp[3], const double Sp[3], const double Sm[3], double G[4]) {
  double ep = delta * omega, em = (1.0 - delta) * omega, eg = omega;
  double rho = 2.0 / (3.0 * chig * delta * (1.0 - delta));
  double ks[3];
  or_ktable(c, rho, ks);
  double K13 = ks[0], K23 = ks[1], IK = ks[2];
  double epm = em * ep;
  double sum2 = (em * em + ep * ep) / epm, dif2 = (ep * ep - em * em) / epm, sq = (ep - em) * (ep - em) / epm;
  double SpSm = dot3(Sp, Sm);
  double Spb = dot3(Sp, bp), Smb = dot3(Sm, bp), Spa = dot3(Sp, ap), Sma = dot3(Sm, ap);
  double Spv = dot3(Sp, vp), Smv = dot3(Sm, vp);
  double x[3];
  cross3(Sm, Sp, x);
  G[0] = IK + sum2 * K23 + (IK - 2 * K23) * SpSm + K13 * (-(eg / ep) * Spb + (eg / em) * Smb) +
         (sum2 * IK - sq * K23) * Spv * Smv;
  G[1] = K13 * (-(eg / em) * Spa + (eg / ep) * Sma) + 0.5 * dif2 * K23 * dot3(x, vp) -
         (eg * eg / (2 * epm)) * IK * (Spa * Smb + Sma * Spb);
  G[2] = (eg * eg / (2 * epm)) * K13 * dot3(x, ap) + 0.5 * dif2 * K13 * (Smv * Spb + Spv * Smb) +
         ((eg / em) * IK - dif2 * K23) * Smv + ((eg / ep) * IK + dif2 * K23) * Spv;
  G[3] = -K23 + 0.5 * sum2 * K23 * SpSm - K13 * ((eg / ep) * Smb - (eg / em) * Spb) +
         (eg * eg / (2 * epm)) * IK * (Spb * Smb - Spa * Sma) - 0.5 * sq * K23 * Spv * Smv;
}

/* ======================================================================= *
 *  High-energy bremsstrahlung and Bethe-Heitler pair production in matter *
 *  (Sec. III E).                                                           *
 *  Differential cross-sections of Tsai (Rev. Mod. Phys. 46, 815 (1974)):   *
 *    brems:  dsigma/dy = alpha r0^2 D_b / y, y = omega / E,                *
 *      D_b = (4/3 - 4/3 y + y^2) A + (2/3)(1 - y) B          (the paper's  *
 *      printed cross-section),                                             *
 *    pairs:  dsigma/dx = alpha r0^2 D_p, x = E+ / k,                       *
 *      D_p = (1 - 4/3 x(1-x)) A - (2/3) x(1-x) B   (the same amplitudes    *
 *      with the pair's energies: E^2 + E'^2 - 2/3 E E' -> E+^2 + E-^2 +    *
 *      2/3 E+ E-, the paper's "similar process"),                          *
 *    A = Z^2 (phi1 - 4/3 ln Z - 4 f) + Z (psi1 - 8/3 ln Z),                *
 *    B = Z^2 (phi1 - phi2) + Z (psi1 - psi2),                              *
 *  with Tsai's screening functions phi1,2(gamma), psi1,2(eps) (his Eqs.    *
 *  3.38-3.41, Thomas-Fermi atoms, Z >= 5), gamma = 100 m k/(E E' Z^1/3),   *
 *  eps = 100 m k/(E E' Z^2/3), and the Coulomb correction f(Z).  D < 0,    *
 *  where the fits leave their range (no screening, near the end points),   *
 *  is taken as 0.                                                           *
 *  Event per step (Sec. III E): P = 1 - exp(-n sigma(E) ds), ds = v dt;    *
 *  energy fraction from r sigma(E) = sigma(y, E) (cumulative).  Tables     *
 *  (a specification shared with the GPU path): rows at NMG energies, ln E  *
 *  uniform on [ln 2, ln 2e6] (m c^2); each row the cumulative integral at  *
 *  NMS nodes of s in [0, 1], s uniform in ln(v/(1-v)) from v_lo to v_hi    *
 *  (brems v = y in [k_min/E, 1 - 1/E], pairs v = x in [1/k, 1 - 1/k]),     *
 *  each node interval by 8-point Gauss-Legendre.                           *
 * ======================================================================= */
void or_screening(double g, double e, double out[4]) {
  out[0] = 20.863 - 2.0 * log(1.0 + (0.55846 * g) * (0.55846 * g)) -
           4.0 * (1.0 - 0.6 * exp(-0.9 * g) - 0.4 * exp(-1.5 * g));
  out[1] = out[0] - (2.0 / 3.0) / (1.0 + 6.5 * g + 6.0 * g * g);
  out[2] = 28.340 - 2.0 * log(1.0 + (3.621 * e) * (3.621 * e)) -
           4.0 * (1.0 - 0.7 * exp(-8.0 * e) - 0.3 * exp(-29.2 * e));
  out[3] = out[2] - (2.0 / 3.0) / (1.0 + 40.0 * e + 400.0 * e * e);
}

double or_coulomb_f(int Z) {
  double a2 = (OR_ALPHA * Z) * (OR_ALPHA * Z);
  return a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
}

/* A and B at screening argument d = m k/(E E') */
static void or_med_AB(int Z, double d, double *A, double *B) {
  double z13 = cbrt((double)Z), lz = log((double)Z), s[4];
  or_screening(100.0 * d / z13, 100.0 * d / (z13 * z13), s);
  double f = or_coulomb_f(Z), z2 = (double)Z * Z;
  *A = z2 * (s[0] - 4.0 / 3.0 * lz - 4.0 * f) + Z * (s[2] - 8.0 / 3.0 * lz);
  *B = z2 * (s[0] - s[1]) + Z * (s[2] - s[3]);
}

double or_brems_D(int Z, double E, double y) {
  if (!(y > 0.0) || !(y < 1.0)) return 0.0;
  double A, B;
  or_med_AB(Z, y / (E * (1.0 - y)), &A, &B);
  double D = (4.0 / 3.0 - 4.0 / 3.0 * y + y * y) * A + (2.0 / 3.0) * (1.0 - y) * B;
  return D > 0.0 ? D : 0.0;
}

double or_pair_D(int Z, double k, double x) {
  if (!(x > 0.0) || !(x < 1.0)) return 0.0;
  double A, B, xx = x * (1.0 - x);
  or_med_AB(Z, 1.0 / (k * xx), &A, &B);
  double D = (1.0 - 4.0 / 3.0 * xx) * A - (2.0 / 3.0) * xx * B;
  return D > 0.0 ? D : 0.0;
}

/* the variable of coordinate s of a row at energy E (which: 0 brems y, 1 pairs x) and the
   Jacobian of the cross-section in s.  s is uniform in t = ln(v / (1 - v)) between the
   end points v_lo and v_hi: logarithmic at both ends (y -> k_min/E, y -> 1 - 1/E;
   x -> 1/k, x -> 1 - 1/k), where the braces vary fastest.  With dv = v (1 - v) dt:
   brems D/y dy = D (1 - y) dt, pairs D dx = D x (1 - x) dt. */
static double or_med_var(int which, double E, double kmin, double s, double *jac) {
  double vlo = which == 0 ? kmin / E : 1.0 / E, vhi = 1.0 - 1.0 / E;
  double tlo = log(vlo / (1.0 - vlo)), thi = log(vhi / (1.0 - vhi));
  double t = tlo + s * (thi - tlo);
  double v = 1.0 / (1.0 + exp(-t)), w = 1.0 / (1.0 + exp(t));   /* v and 1 - v */
  *jac = (thi - tlo) * (which == 0 ? w : v * w);
  return v;
}

/* cumulative table of one process: C[i][j] = integral over s in [0, s_j] */
static void or_build_medium(int Z, double kmin, int which, double *C) {
  double hE = (MG_HI - MG_LO) / (NMG - 1), hs = 1.0 / (NMS - 1);
  for (int i = 0; i < NMG; ++i) {
    double E = exp(MG_LO + i * hE);
    double *row = C + (size_t)i * NMS;
    row[0] = 0.0;
    int open = which == 0 ? (kmin / E < 1.0 - 1.0 / E) : (E > 2.0);
    for (int j = 1; j < NMS; ++j) {
      double acc = 0.0;
      if (open) {
        for (int q = 0; q < 8; ++q) {
          double s = (j - 1) * hs + 0.5 * hs * (GL8X[q] + 1.0), jac;
          double v = or_med_var(which, E, kmin, s, &jac);
          double D = which == 0 ? or_brems_D(Z, E, v) : or_pair_D(Z, E, v);
          acc += GL8W[q] * D * jac;
        }
        acc *= 0.5 * hs;
      }
      row[j] = row[j - 1] + acc;
    }
  }
}

void or_set_medium(or_ctx *c, const or_medium *m) {
  if (!m) { c->has_medium = 0; return; }
  c->med = *m;
  or_build_medium(m->Z, m->k_min, 0, &c->mb[0][0]);
  or_build_medium(m->Z, m->k_min, 1, &c->mp[0][0]);
  c->has_medium = 1;
}

/* row interpolation of a table at ln E: the total sigma(E) (returned) and, for r in [0,1),
   the node coordinate s with (1-w) C_i(s) + w C_i+1(s) = r sigma(E) (piecewise linear) */
static double or_med_lookup(const double *C, double lnE, double r, double *s_out, int *range) {
  double t = (lnE - MG_LO) / ((MG_HI - MG_LO) / (NMG - 1));
  if (t > NMG - 1) { t = NMG - 1; if (range) *range = 1; }
  if (t < 0) return 0.0;
  int i = (int)floor(t);
  if (i > NMG - 2) i = NMG - 2;
  double w = t - i;
  const double *a = C + (size_t)i * NMS, *b = a + NMS;
  double tot = (1.0 - w) * a[NMS - 1] + w * b[NMS - 1];
  if (s_out && tot > 0.0) {
    double target = r * tot;
    int lo = 0, hi = NMS - 1;
    while (hi - lo > 1) {
      int mid = (lo + hi) / 2;
      double cm = (1.0 - w) * a[mid] + w * b[mid];
      if (cm <= target) lo = mid; else hi = mid;
    }
    double c0 = (1.0 - w) * a[lo] + w * b[lo], c1 = (1.0 - w) * a[lo + 1] + w * b[lo + 1];
    double f = c1 > c0 ? (target - c0) / (c1 - c0) : 0.0;
    *s_out = (lo + f) / (NMS - 1);
  }
  return tot;
}

double or_medium_sigma(const or_ctx *c, int which, double E) {
  if (!c->has_medium || !(E > 0.0)) return 0.0;
  return or_med_lookup(which == 0 ? &c->mb[0][0] : &c->mp[0][0], log(E), 0.0, NULL, NULL);
}

/* the sampled variable (y or x) for energy E and uniform r */
double or_medium_sample(const or_ctx *c, int which, double E, double r) {
  double s = 0.0, jac;
  or_med_lookup(which == 0 ? &c->mb[0][0] : &c->mp[0][0], log(E), r, &s, NULL);
  return or_med_var(which, E, c->med.k_min, s, &jac);
}

static int or_in_medium(const or_ctx *c, const double x[3]) {
  double v = x[c->med.axis];
  return v >= c->med.lo && v < c->med.hi;
}

/* ======================================================================= *
 *  Birth records                                                           *
 * ======================================================================= */
typedef struct { double x[3], p[3], s[3], w; } or_lep_birth;
typedef struct { double x[3], k[3], xi[3], th, w; } or_ph_birth;

/* Near-tie log: every discrete decision "r < thr" of a step (r a uniform draw, thr its
 * threshold) whose draw lies within near_tol relative of the threshold, |r - thr| < near_tol
 * thr, is recorded as (id, step, kind, |r - thr|/thr).  A second implementation that
 * computes thr with rounding errors of relative size e can take a different branch only
 * where this margin is below e. */
static void or_note(or_ctx *c, uint64_t id, uint32_t step, uint32_t kind, double r, double thr, or_stats *st) {
  if (!(thr > 0.0)) return;
  double m = fabs(r - thr) / thr;
  if (m < c->near_tol) {
    if (st) st->n_near++;
#ifdef _OPENMP
#pragma omp critical(or_near_log)
#endif
    {
      if (c->nlog < c->logcap) {
        c->log_id[c->nlog] = id; c->log_step[c->nlog] = step; c->log_kind[c->nlog] = kind;
        c->log_margin[c->nlog] = m;
      }
      c->nlog++;
    }
  }
}

/* ======================================================================= *
 *  Photon step: frame rotation ROT(psi) (Eq. rotation), VB QED(dphi)       *
 *  (Eq. rotation2, Algorithm "VB effect in SLIPs"), NBW decision and pair  *
 *  sampling (Sec. III D MC algorithm).  Returns 1 if the photon decayed.   *
 * ======================================================================= */
static int or_photon(or_ctx *c, or_particles *ph, uint64_t i, const or_fields *f, double t, double dt,
                     uint64_t seed, uint32_t step, uint32_t flags, or_lep_birth *be, or_lep_birth *bp,
                     or_stats *st) {
  double x[3] = {ph->x[i], ph->y[i], ph->z[i]};
  double k[3] = {ph->px[i], ph->py[i], ph->pz[i]};
  double xi[3] = {ph->s1[i], ph->s2[i], ph->s3[i]};
  double th = ph->theta[i];
  double E[3], B[3];
  or_field(f, x[0], x[1], x[2], t, E, B);
  double om = norm3(k);
  double n[3] = {k[0] / om, k[1] / om, k[2] / om};
  double ne = dot3(n, E), nxB[3];
  cross3(n, B, nxB);
  double Er[3] = {E[0] - n[0] * ne + nxB[0], E[1] - n[1] * ne + nxB[1], E[2] - n[2] * ne + nxB[2]};
  double er = norm3(Er);
  int decayed = 0;
  if (er > 0.0 && (flags & (OR_F_VB | OR_F_NBW))) {
    double chig = OR_XIL * om * er;
    double P1[3] = {Er[0] / er, Er[1] / er, Er[2] / er}, P2[3];
    cross3(n, P1, P2);
    double e1[3], e2[3];
    or_frame(n, e1, e2);
    double thn = atan2(dot3(P1, e2), dot3(P1, e1));
    double psi = thn - th;
    double c2 = cos(2 * psi), s2 = sin(2 * psi);
    double x1 = xi[0] * c2 - xi[2] * s2, x3 = xi[0] * s2 + xi[2] * c2;
    xi[0] = x1; xi[2] = x3;
    th = thn;
    if (flags & OR_F_VB) {
      double M[2];
      double cv = chig > OR_VB_MAX ? OR_VB_MAX : chig;
      or_vb_m(c, cv, M);
      double dphi = (M[0] - M[1]) * (OR_ALPHA / (90.0 * OR_PI)) * OR_XIL * om * er * er * dt;
      double cd = cos(dphi), sd = sin(dphi);
      double y1 = cd * xi[0] - sd * xi[1], y2 = sd * xi[0] + cd * xi[1];
      xi[0] = y1; xi[1] = y2;
    }
    if ((flags & OR_F_NBW) && om >= 2.0 && chig >= OR_CHIG_MIN) {
      double cg = chig;
      if (cg > OR_CHIG_MAX) { cg = OR_CHIG_MAX; if (st) st->n_range++; }
      double T[2];
      or_nbw_rates(c, cg, T);
      double P = OR_ALPHA / (sqrt(3.0) * OR_PI * OR_XIL * om) * (T[0] - xi[2] * T[1]) * dt;
      double r[2];
      or_uniforms(seed, ph->id[i], step, 3u, r);
      or_note(c, ph->id[i], step, OR_D_NBW, r[0], P, st);
      /* one event per particle per step (reading of the independence of events within a
         step): count the decisions where that is coarse */
      if (P > 0.1 && st) st->n_coarse++;
      if (r[0] < P) {
        /* energy split: mixture over xi3' = +-1 components */
        double w0 = 0.5 * (1.0 + xi[2]) * (T[0] - T[1]);
        int comp = (r[1] * (T[0] - xi[2] * T[1]) < w0) ? 0 : 1;
        or_note(c, ph->id[i], step, OR_D_NBW_COMP, r[1], w0 / (T[0] - xi[2] * T[1]), st);
        double r2[2];
        or_uniforms(seed, ph->id[i], step, 4u, r2);
        double l = r2[0];
        int upper = l >= 0.5;
        double lam = upper ? 2.0 * (1.0 - l) : 2.0 * l;
        double tt = lam > 0 ? log(lam) : BT_LO;
        if (tt < BT_LO) tt = BT_LO;
        double dh = exp(or_nbw_invcdf(c, comp, cg, tt));
        double ep = upper ? (1.0 - dh) * om : dh * om;
        if (ep < 1.0) ep = 1.0;
        if (ep > om - 1.0) ep = om - 1.0;
        double em = om - ep;
        double delta = ep / om;
        /* SQAs: S+ along D (Eq. BWposAxis2), S- along D' (Eq. BWeleAxis1);
           a+ = P1', b+ = n x a+ = P2', v+ = n */
        double rho = 2.0 / (3.0 * cg * delta * (1.0 - delta));
        double ks[3];
        or_ktable(c, rho, ks);
        double K13 = ks[0], K23 = ks[1], IK = ks[2];
        double dif2 = (ep * ep - em * em) / (ep * em);
        double cb = -(om / ep - xi[2] * om / em) * K13, ca = -xi[0] * (om / em) * K13;
        double cv2 = xi[1] * (dif2 * K23 + (om / ep) * IK);
        double D[3], Dp[3];
        for (int q = 0; q < 3; ++q) D[q] = cb * P2[q] + ca * P1[q] + cv2 * n[q];
        double cbp = (om / em - xi[2] * om / ep) * K13, cap = xi[0] * (om / ep) * K13;
        double cvp = -xi[1] * (dif2 * K23 - (om / em) * IK);
        for (int q = 0; q < 3; ++q) Dp[q] = cbp * P2[q] + cap * P1[q] + cvp * n[q];
        double dn = norm3(D), dpn = norm3(Dp);
        double Sp[3], Sm[3];
        for (int q = 0; q < 3; ++q) {
          Sp[q] = dn > 0 ? D[q] / dn : P2[q];
          Sm[q] = dpn > 0 ? Dp[q] / dpn : P2[q];
        }
        double Pk[4], tot = 0;
        for (int o = 0; o < 4; ++o) {
          double sp = (o < 2) ? 1.0 : -1.0, sm = (o % 2 == 0) ? 1.0 : -1.0;
          double a1[3] = {sp * Sp[0], sp * Sp[1], sp * Sp[2]}, a2[3] = {sm * Sm[0], sm * Sm[1], sm * Sm[2]};
          double G[4];
          or_nbw_G(c, delta, om, cg, P1, P2, n, a1, a2, G);
          Pk[o] = G[0] + xi[0] * G[1] + xi[1] * G[2] + xi[2] * G[3];
          if (Pk[o] < 0) Pk[o] = 0;
          tot += Pk[o];
        }
        double rr = r2[1] * tot, acc = 0;
        int o = 3;
        for (int q = 0; q < 4; ++q) {
          acc += Pk[q];
          if (rr < acc) { o = q; break; }
        }
        double cum = 0;
        for (int q = 0; q < 3; ++q) {   /* the three cumulative thresholds of the pick */
          cum += Pk[q];
          or_note(c, ph->id[i], step, OR_D_NBW_SPIN, r2[1], cum / tot, st);
        }
        double sp = (o < 2) ? 1.0 : -1.0, sm = (o % 2 == 0) ? 1.0 : -1.0;
        double pp = sqrt(ep * ep - 1.0), pm = sqrt(em * em - 1.0);
        for (int q = 0; q < 3; ++q) {
          bp->x[q] = x[q]; be->x[q] = x[q];
          bp->p[q] = pp * n[q]; be->p[q] = pm * n[q];
          bp->s[q] = sp * Sp[q]; be->s[q] = sm * Sm[q];
        }
        bp->w = be->w = ph->w[i];
        decayed = 1;
        if (st) st->n_nbw++;
      }
    }
  }
  /* Bethe-Heitler pair creation in matter (Sec. III E), if the photon did not decay by
     NBW: P = 1 - exp(-n sigma(k) c dt), the positron's energy fraction x from the
     cumulative cross-section; the pair moves along the photon, born at its x^n.  The
     pair's spins are not resolved: S = 0, the unpolarised (mixed) state. */
  if (!decayed && (flags & OR_F_BH) && c->has_medium && om > 2.0 && or_in_medium(c, x)) {
    int range = 0;
    double sig = or_med_lookup(&c->mp[0][0], log(om), 0.0, NULL, &range);
    if (range && st) st->n_range++;
    double P = -expm1(-c->med.n * OR_ALPHA * OR_R0N * OR_R0N * sig * dt);
    double r[2];
    or_uniforms(seed, ph->id[i], step, 6u, r);
    or_note(c, ph->id[i], step, OR_D_BH, r[0], P, st);
    if (P > 0.1 && st) st->n_coarse++;
    if (r[0] < P) {
      double xf = or_medium_sample(c, 1, om, r[1]);
      double ep = xf * om;
      if (ep < 1.0) ep = 1.0;
      if (ep > om - 1.0) ep = om - 1.0;
      double em = om - ep;
      double pp = sqrt(ep * ep - 1.0), pm = sqrt(em * em - 1.0);
      for (int q = 0; q < 3; ++q) {
        bp->x[q] = x[q]; be->x[q] = x[q];
        bp->p[q] = pp * n[q]; be->p[q] = pm * n[q];
        bp->s[q] = 0.0; be->s[q] = 0.0;
      }
      bp->w = be->w = ph->w[i];
      decayed = 1;
      if (st) st->n_bh++;
    }
  }
  if (!decayed) {
    for (int q = 0; q < 3; ++q) x[q] += dt * n[q];
    ph->x[i] = x[0]; ph->y[i] = x[1]; ph->z[i] = x[2];
    ph->s1[i] = xi[0]; ph->s2[i] = xi[1]; ph->s3[i] = xi[2];
    ph->theta[i] = th;
  }
  return decayed;
}

/* ======================================================================= *
 *  Lepton step: Boris push (Eqs. boris1-boris6), T-BMT by Boris rotation   *
 *  (Eqs. bmteqn, bmt-boris1..4), position (Eq. lorentz2), chi_e (Sec. III *
 *  A), NCS decision / no-emission spin update + collapse / emission with  *
 *  recoil, spin collapse and photon Stokes (Sec. III C MC procedure).     *
 *  Returns 1 if a photon was emitted.                                      *
 * ======================================================================= */
static int or_lepton(or_ctx *c, or_particles *L, uint64_t i, double q, const or_fields *f, double t, double dt,
                     uint64_t seed, uint32_t step, uint32_t flags, or_ph_birth *bph, or_stats *st, int species) {
  double x[3] = {L->x[i], L->y[i], L->z[i]};
  double p0[3] = {L->px[i], L->py[i], L->pz[i]};
  double S[3] = {L->s1[i], L->s2[i], L->s3[i]};
  double E[3], B[3];
  or_field(f, x[0], x[1], x[2], t, E, B);
  /* Boris */
  double hq = 0.5 * q * dt;
  double pm[3] = {p0[0] + hq * E[0], p0[1] + hq * E[1], p0[2] + hq * E[2]};
  double gm = sqrt(1.0 + dot3(pm, pm));
  double tau[3] = {hq * B[0] / gm, hq * B[1] / gm, hq * B[2] / gm};
  double pxt[3], pp[3];
  cross3(pm, tau, pxt);
  for (int k = 0; k < 3; ++k) pp[k] = pm[k] + pxt[k];
  double sfac = 2.0 / (1.0 + dot3(tau, tau));
  double sig[3] = {sfac * tau[0], sfac * tau[1], sfac * tau[2]};
  double ppxs[3];
  cross3(pp, sig, ppxs);
  double pn[3];
  for (int k = 0; k < 3; ++k) pn[k] = pm[k] + ppxs[k] + hq * E[k];
  /* Radiative pusher (Sec. III A "Algorithms of the Radiative Pusher" and Sec. III B
   * radiative T-BMT).  Readings: the radiation force and the radiative spin term are
   * evaluated once, at time n, with the fields at x^n and the time-centred momentum
   * pb = (p^{n-1/2} + p_L^{n+1/2})/2 of the Boris step; the LL force keeps the second and
   * third terms of Eq. eq1-1 (the field-derivative term is dropped: the paper notes the
   * last two dominate in ultra-intense fields) with 1/gamma restored on E(p.E) as in
   * Eq. eq1; the third term is written through chi: gamma p[(E+beta x B)^2-(beta.E)^2] =
   * chi^2 beta / xi_L^2; n_B = beta x a is taken as the unit vector n x a. */
  double rs_P = 0, rs_psi[3] = {0, 0, 0}, rs_be[3] = {0, 0, 0}, rs_z[3] = {0, 0, 0};
  int rs_on = 0;
  if (flags & (OR_F_LL | OR_F_MLL | OR_F_MBMT)) {
    double pb[3] = {0.5 * (p0[0] + pn[0]), 0.5 * (p0[1] + pn[1]), 0.5 * (p0[2] + pn[2])};
    double gb = sqrt(1.0 + dot3(pb, pb));
    double pbm = norm3(pb);
    double be[3] = {pb[0] / gb, pb[1] / gb, pb[2] / gb};
    double chi = 0.0, v[3] = {0, 0, 0}, vm = 0.0, nb[3] = {0, 0, 0};
    if (pbm > 0.0) {
      for (int k = 0; k < 3; ++k) nb[k] = pb[k] / pbm;
      double nE = dot3(nb, E), pxB[3];
      cross3(pb, B, pxB);
      for (int k = 0; k < 3; ++k) v[k] = gb * (E[k] - nb[k] * nE) + pxB[k];
      vm = norm3(v);
      chi = OR_XIL * sqrt(vm * vm + nE * nE);
    }
    double chit = chi;
    if (chit > OR_CHI_MAX) { chit = OR_CHI_MAX; if (st) st->n_range++; }
    double fn[4] = {1.0, 0, 0, 0};
    if (chit > 0.0) or_rr_funcs(c, chit, fn);
    if (flags & (OR_F_LL | OR_F_MLL)) {
      double qf = (flags & OR_F_MLL) ? fn[0] : 1.0;
      double ExB[3], Bxp[3], BxBxp[3];
      cross3(E, B, ExB);
      cross3(B, pb, Bxp);
      cross3(B, Bxp, BxBxp);
      double pE = dot3(pb, E);
      double c2 = 2.0 / 3.0 * OR_ALPHA * OR_XIL, c3 = 2.0 / 3.0 * OR_ALPHA / OR_XIL * chi * chi;
      for (int k = 0; k < 3; ++k) {
        double F = qf * (c2 * (ExB[k] + BxBxp[k] / gb + E[k] * pE / gb) - c3 * be[k]);
        pn[k] += F * dt;
      }
    }
    if ((flags & OR_F_MBMT) && vm > 0.0 && chi > 0.0) {
      double sq = q > 0 ? 1.0 : -1.0;
      double a[3] = {sq * v[0] / vm, sq * v[1] / vm, sq * v[2] / vm};
      cross3(nb, a, rs_z);
      rs_P = OR_ALPHA / (sqrt(3.0) * OR_PI * gb * OR_XIL);
      for (int k = 0; k < 3; ++k) { rs_psi[k] = fn[k + 1]; rs_be[k] = be[k]; }
      rs_on = 1;
    }
  }
  /* radiative T-BMT half kick: S += dt/2 (dS/dt)_R, (dS/dt)_R = -P[psi1 S + psi2 (S.beta)
   * beta + psi3 n_B] (Eq. spin1) */
  if (rs_on) {
    double sb = dot3(S, rs_be);
    for (int k = 0; k < 3; ++k)
      S[k] += 0.5 * dt * (-rs_P * (rs_psi[0] * S[k] + rs_psi[1] * sb * rs_be[k] + rs_psi[2] * rs_z[k]));
  }
  /* T-BMT (reading: beta, gamma from the mean of p^{n-1/2}, p^{n+1/2};
     dS/dt = q S x Omega as implied by t = q dt Omega / 2) */
  if (flags & OR_F_SPIN) {
    double pa[3] = {0.5 * (p0[0] + pn[0]), 0.5 * (p0[1] + pn[1]), 0.5 * (p0[2] + pn[2])};
    double ga = sqrt(1.0 + dot3(pa, pa));
    double be[3] = {pa[0] / ga, pa[1] / ga, pa[2] / ga};
    double bB = dot3(be, B), bxE[3];
    cross3(be, E, bxE);
    double c1 = -OR_AE * ga / (ga + 1.0) * bB;
    double c2 = OR_AE + 1.0 / ga;
    double c3 = -(OR_AE + 1.0 - ga / (ga + 1.0));
    double Om[3];
    for (int k = 0; k < 3; ++k) Om[k] = c1 * be[k] + c2 * B[k] + c3 * bxE[k];
    double tv[3] = {hq * Om[0], hq * Om[1], hq * Om[2]};
    double of = 2.0 / (1.0 + dot3(tv, tv));
    double ov[3] = {of * tv[0], of * tv[1], of * tv[2]};
    double sxt[3], S1[3], s1xo[3];
    cross3(S, tv, sxt);
    for (int k = 0; k < 3; ++k) S1[k] = S[k] + sxt[k];
    cross3(S1, ov, s1xo);
    for (int k = 0; k < 3; ++k) S[k] += s1xo[k];
  }
  if (rs_on) {
    double sb = dot3(S, rs_be);
    for (int k = 0; k < 3; ++k)
      S[k] += 0.5 * dt * (-rs_P * (rs_psi[0] * S[k] + rs_psi[1] * sb * rs_be[k] + rs_psi[2] * rs_z[k]));
  }
  /* position with the pre-QED p^{n+1/2} (after the radiation force when it is on) */
  double g1 = sqrt(1.0 + dot3(pn, pn));
  double xo[3] = {x[0], x[1], x[2]};
  for (int k = 0; k < 3; ++k) x[k] += dt * pn[k] / g1;
  /* current of the move x^n -> x^{n+1} (Sec. II C), with v_z of the same p^{n+1/2} */
  if ((flags & OR_F_DEPOSIT) && f->kind == OR_FIELD_GRID2D && f->gJx)
    or_deposit(f, q * L->w[i], xo, x, pn[2] / g1, dt);
  int emitted = 0, ncs_event = 0;
  if (flags & OR_F_NCS) {
    double pmag = norm3(pn);
    if (pmag <= 0.0) pmag = 1e-300;   /* at rest: chi = 0 below, no QED */
    double n[3] = {pn[0] / pmag, pn[1] / pmag, pn[2] / pmag};
    double nE = dot3(n, E), pxB[3];
    cross3(pn, B, pxB);
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = g1 * (E[k] - n[k] * nE) + pxB[k];
    double vm = norm3(v);
    double chi = OR_XIL * sqrt(vm * vm + nE * nE);
    if (chi >= OR_CHI_MIN && vm > 0.0) {
      if (chi > OR_CHI_MAX) { chi = OR_CHI_MAX; if (st) st->n_range++; }
      double sq = q > 0 ? 1.0 : -1.0;
      double a[3] = {sq * v[0] / vm, sq * v[1] / vm, sq * v[2] / vm};
      double z[3];
      cross3(n, a, z);
      double AB[2];
      or_ncs_rates(c, chi, AB);
      double s = dot3(S, z);
      double pref = OR_ALPHA / (sqrt(3.0) * OR_PI * OR_XIL * g1);
      double Wa = pref * AB[0], Wb = pref * AB[1];
      double P = (Wa - s * Wb) * dt;
      double r[2];
      or_uniforms(seed, L->id[i], step, 0u, r);
      or_note(c, L->id[i], step, OR_D_NCS, r[0], P, st);
      if (P > 0.1 && st) st->n_coarse++;
      if (r[0] < P) {
        double rm[2], rs[2];
        or_uniforms(seed, L->id[i], step, 1u, rm);
        or_uniforms(seed, L->id[i], step, 2u, rs);
        /* photon energy: exact two-component mixture of Eq. Wspin2 at s = S.zeta */
        double wplus = 0.5 * (1.0 + s) * (AB[0] - AB[1]);
        int comp = (rm[0] * (AB[0] - s * AB[1]) < wplus) ? 0 : 1;
        or_note(c, L->id[i], step, OR_D_NCS_COMP, rm[0], wplus / (AB[0] - s * AB[1]), st);
        double l = rm[1];
        double tt = (l > 0.0) ? log(l) - log1p(-l) : CT_LO;
        if (tt < CT_LO) tt = CT_LO;
        if (tt > CT_HI) tt = CT_HI;
        double u = exp(or_ncs_invcdf(c, comp, chi, tt));
        double omr = 1.0 / (1.0 + u), rr = u / (1.0 + u);
        double om = rr * g1;
        /* emission spin: SQA from F0 as a linear function of S_f (Eq. F0);
           P(+) = (1 + |g|/c0)/2.  F0 = c0 + g.S_f is affine in S_f; g_k is read off as
           (F0(L e_k) - F0(-L e_k)) / 2L with L = 2^30, where c0 cancels exactly: with a
           unit S_f the difference F0(e_k) - c0 would carry the rounding of c0, which for
           an unpolarised lepton (S_i = 0, |g| ~ u c0) and a soft photon is ~1e-16/u of
           |g| in the direction of the axis */
        double F[4], Fp[4], Fm[4];
        const double Lb = 1073741824.0;
        double mz[3] = {0, 0, 0};
        or_ncs_F(c, u, chi, n, a, S, mz, F);
        double c0 = F[0];
        double g[3];
        for (int k = 0; k < 3; ++k) {
          double ep[3] = {0, 0, 0}, em[3] = {0, 0, 0};
          ep[k] = Lb; em[k] = -Lb;
          or_ncs_F(c, u, chi, n, a, S, ep, Fp);
          or_ncs_F(c, u, chi, n, a, S, em, Fm);
          g[k] = (Fp[0] - Fm[0]) / (2.0 * Lb);
        }
        double gm2 = norm3(g);
        double Sf[3];
        if (gm2 > 0.0) {
          double sgn = (rs[0] < 0.5 * (1.0 + gm2 / c0)) ? 1.0 : -1.0;
          or_note(c, L->id[i], step, OR_D_NCS_SPIN, rs[0], 0.5 * (1.0 + gm2 / c0), st);
          for (int k = 0; k < 3; ++k) Sf[k] = sgn * g[k] / gm2;
        } else {
          for (int k = 0; k < 3; ++k) Sf[k] = S[k];
        }
        /* photon Stokes: pure states +-F/|F| (F = F1..F3 at chosen S_f) */
        or_ncs_F(c, u, chi, n, a, S, Sf, F);
        double fm = sqrt(F[1] * F[1] + F[2] * F[2] + F[3] * F[3]);
        double xi[3] = {0, 0, 0};
        if (fm > 0.0) {
          double sg = (rs[1] < 0.5 * (1.0 + fm / F[0])) ? 1.0 : -1.0;
          or_note(c, L->id[i], step, OR_D_NCS_STOKES, rs[1], 0.5 * (1.0 + fm / F[0]), st);
          for (int k = 0; k < 3; ++k) xi[k] = sg * F[k + 1] / fm;
        }
        for (int k = 0; k < 3; ++k) S[k] = Sf[k];
        if (!(flags & OR_F_NO_RECOIL)) {
          /* recoil: p_f = p_i - omega n (reading: omega = r gamma, momentum conserved),
             |p_f| = (1-r) gamma - (gamma - |p|) without cancellation */
          double pf = omr * g1 - 1.0 / (g1 + pmag);
          for (int k = 0; k < 3; ++k) pn[k] = pf * n[k];
          if (!(flags & OR_F_DROP_PHOTONS)) {
            double e1[3], e2[3];
            or_frame(n, e1, e2);
            for (int k = 0; k < 3; ++k) {
              bph->x[k] = x[k];
              bph->k[k] = om * n[k];
              bph->xi[k] = xi[k];
            }
            bph->th = atan2(dot3(a, e2), dot3(a, e1));
            bph->w = L->w[i];
            emitted = 1;
          }
        }
        if (st) st->n_ncs[species]++;
        ncs_event = 1;
      } else {
        /* no emission: posterior mean spin (reading: W and f are u-integrated,
           f = -Wb zeta), then collapse with P(+) = (1 + |S|)/2 */
        double den = 1.0 - P;
        double Sb[3];
        for (int k = 0; k < 3; ++k) Sb[k] = (S[k] * (1.0 - Wa * dt) + Wb * dt * z[k]) / den;
        double m = norm3(Sb);
        double sg = (r[1] < 0.5 * (1.0 + m)) ? 1.0 : -1.0;
        or_note(c, L->id[i], step, OR_D_NCS_COLLAPSE, r[1], 0.5 * (1.0 + m), st);
        for (int k = 0; k < 3; ++k) S[k] = sg * Sb[k] / m;
      }
    }
  }
  /* Bremsstrahlung in matter (Sec. III E), if no NCS event this step (one event per
     particle per step): P = 1 - exp(-n sigma(E) v dt) at the energy of p^{n+1/2} and the
     position x^n; photon energy omega = y E from the cumulative cross-section, along p;
     the lepton keeps its direction with energy E - omega (the nucleus takes the
     momentum balance); the photon is unpolarised (xi = 0) and born at x^{n+1}; the
     lepton spin is not changed (the process is not spin-resolved). */
  if (!ncs_event && (flags & OR_F_BREMS) && c->has_medium && or_in_medium(c, xo)) {
    int range = 0;
    double pmag = norm3(pn);
    double sig = or_med_lookup(&c->mb[0][0], log(g1), 0.0, NULL, &range);
    if (range && st) st->n_range++;
    double P = -expm1(-c->med.n * OR_ALPHA * OR_R0N * OR_R0N * sig * (pmag / g1) * dt);
    double r[2];
    or_uniforms(seed, L->id[i], step, 5u, r);
    or_note(c, L->id[i], step, OR_D_BREMS, r[0], P, st);
    if (P > 0.1 && st) st->n_coarse++;
    if (r[0] < P && pmag > 0.0) {
      double yv = or_medium_sample(c, 0, g1, r[1]);
      double om = yv * g1;
      double gf = g1 - om;
      if (gf < 1.0) gf = 1.0;
      double nv[3] = {pn[0] / pmag, pn[1] / pmag, pn[2] / pmag};
      if (!(flags & OR_F_NO_RECOIL)) {
        double pf = sqrt(gf * gf - 1.0);
        for (int k = 0; k < 3; ++k) pn[k] = pf * nv[k];
        if (!(flags & OR_F_DROP_PHOTONS)) {
          for (int k = 0; k < 3; ++k) {
            bph->x[k] = x[k];
            bph->k[k] = om * nv[k];
            bph->xi[k] = 0.0;
          }
          bph->th = 0.0;
          bph->w = L->w[i];
          emitted = 1;
        }
      }
      if (st) st->n_brems[species]++;
    }
  }
  L->x[i] = x[0]; L->y[i] = x[1]; L->z[i] = x[2];
  L->px[i] = pn[0]; L->py[i] = pn[1]; L->pz[i] = pn[2];
  L->s1[i] = S[0]; L->s2[i] = S[1]; L->s3[i] = S[2];
  return emitted;
}

/* ======================================================================= *
 *  One step, in the order of Sec. IV (VB => NBW for photons, then push,    *
 *  T-BMT and NCS for leptons); newborns are appended and first processed   *
 *  at the next step.  Ids: NBW pairs first (photon order, e- then e+),     *
 *  then NCS photons (e- order, then e+ order).  Decayed photons leave the  *
 *  array: their slots below the new count are refilled from the tail.      *
 *  or_step_decide takes every decision of a step and holds the births;     *
 *  or_step_commit applies them with the ids given (or the sequential ones) *
 * ======================================================================= */
static void or_drop_pending(or_ctx *c) {
  if (!c->pending) return;
  free(c->p_be); free(c->p_bp); free(c->p_bg); free(c->p_dec);
  c->p_be = c->p_bp = c->p_bg = NULL;
  c->p_dec = NULL;
  c->pending = 0;
}

int or_step_decide(or_ctx *c, or_particles *e, or_particles *pos, or_particles *ph, const or_fields *f, double t,
                   double dt, uint64_t seed, uint32_t step, uint32_t flags, or_stats *st, uint64_t counts[3]) {
  or_drop_pending(c);
  uint64_t nph = ph ? ph->n : 0, ne = e ? e->n : 0, np = pos ? pos->n : 0;
  /* every particle's outcome goes to its own slot (index i), so the particle loops may run
     in any order or in parallel; the births are then listed in index order below */
  or_lep_birth *be = (or_lep_birth *)malloc(sizeof(or_lep_birth) * (nph + 1));
  or_lep_birth *bp = (or_lep_birth *)malloc(sizeof(or_lep_birth) * (nph + 1));
  or_ph_birth *bg = (or_ph_birth *)malloc(sizeof(or_ph_birth) * (ne + np + 1));
  unsigned char *dflag = (unsigned char *)calloc(nph + 1, 1);
  unsigned char *eflag = (unsigned char *)calloc(ne + np + 1, 1);
  /* threads: optional, never with deposition (the current sums into one shared grid) */
  int nt = (c->threads > 1 && !(flags & OR_F_DEPOSIT)) ? c->threads : 1;
  or_stats *ts = (or_stats *)calloc((size_t)nt, sizeof(or_stats));
#ifdef _OPENMP
#pragma omp parallel num_threads(nt) if (nt > 1)
#endif
  {
    int me = 0;
#ifdef _OPENMP
    me = omp_get_thread_num();
#endif
    or_stats *mst = st ? &ts[me] : NULL;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
    for (int64_t i = 0; i < (int64_t)nph; ++i)
      dflag[i] = (unsigned char)or_photon(c, ph, (uint64_t)i, f, t, dt, seed, step, flags, &be[i], &bp[i], mst);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
    for (int64_t i = 0; i < (int64_t)(ne + np); ++i) {
      int is_e = i < (int64_t)ne;
      or_particles *L = is_e ? e : pos;
      uint64_t j = is_e ? (uint64_t)i : (uint64_t)i - ne;
      eflag[i] = (unsigned char)or_lepton(c, L, j, is_e ? -1.0 : 1.0, f, t, dt, seed, step, flags, &bg[i], mst,
                                          is_e ? 0 : 1);
    }
  }
  if (st) {
    for (int k = 0; k < nt; ++k) {
      st->n_ncs[0] += ts[k].n_ncs[0]; st->n_ncs[1] += ts[k].n_ncs[1]; st->n_nbw += ts[k].n_nbw;
      st->n_range += ts[k].n_range; st->n_drop += ts[k].n_drop; st->n_near += ts[k].n_near;
      st->n_coarse += ts[k].n_coarse;
      st->n_brems[0] += ts[k].n_brems[0]; st->n_brems[1] += ts[k].n_brems[1]; st->n_bh += ts[k].n_bh;
    }
  }
  free(ts);
  /* decays and emissions in index order: pair births (photon order), NCS photons (e- then
     e+ order) */
  uint64_t nnbw = 0, nncs = 0, nncs_e = 0;
  uint64_t *dec = (uint64_t *)malloc(sizeof(uint64_t) * (nph + 1));
  for (uint64_t i = 0; i < nph; ++i)
    if (dflag[i]) {
      be[nnbw] = be[i]; bp[nnbw] = bp[i];
      dec[nnbw++] = i;
    }
  for (uint64_t i = 0; i < ne + np; ++i)
    if (eflag[i]) {
      bg[nncs++] = bg[i];
      if (i < ne) nncs_e++;
    }
  free(dflag); free(eflag);
  c->pending = 1;
  c->p_be = be; c->p_bp = bp; c->p_bg = bg; c->p_dec = dec;
  c->p_nnbw = nnbw; c->p_nncs = nncs; c->p_nncs_e = nncs_e;
  if (counts) { counts[0] = nnbw; counts[1] = nncs_e; counts[2] = nncs - nncs_e; }
  return 0;
}

int or_step_commit(or_ctx *c, or_particles *e, or_particles *pos, or_particles *ph, const uint64_t *bases,
                   or_stats *st) {
  if (!c->pending) return -1;
  or_lep_birth *be = (or_lep_birth *)c->p_be, *bp = (or_lep_birth *)c->p_bp;
  or_ph_birth *bg = (or_ph_birth *)c->p_bg;
  uint64_t *dec = c->p_dec;
  const uint64_t nnbw = c->p_nnbw, nncs = c->p_nncs, nncs_e = c->p_nncs_e;
  /* the ids: pairs from b[0] (2 a pair), e- emissions from b[1], e+ emissions from b[2];
     the counter continues at b[3].  Alone, they follow one another from next_id. */
  uint64_t b[4];
  if (bases) {
    for (int k = 0; k < 4; ++k) b[k] = bases[k];
  } else {
    b[0] = c->next_id;
    b[1] = b[0] + 2 * nnbw;
    b[2] = b[1] + nncs_e;
    b[3] = b[2] + (nncs - nncs_e);
  }
  /* removal of decayed photons: with M = n - (decays), the k-th decayed slot below M
     receives the k-th surviving photon at or above M (both in index order) */
  if (ph) {
    uint64_t nph = ph->n;
    uint64_t M = nph - nnbw, H = 0;
    while (H < nnbw && dec[H] < M) H++;
    uint64_t q = H, j = M;
    for (uint64_t k = 0; k < H; ++k) {
      while (q < nnbw && dec[q] == j) { q++; j++; }
      uint64_t d = dec[k];
      ph->x[d] = ph->x[j]; ph->y[d] = ph->y[j]; ph->z[d] = ph->z[j];
      ph->px[d] = ph->px[j]; ph->py[d] = ph->py[j]; ph->pz[d] = ph->pz[j];
      ph->s1[d] = ph->s1[j]; ph->s2[d] = ph->s2[j]; ph->s3[d] = ph->s3[j];
      ph->theta[d] = ph->theta[j]; ph->w[d] = ph->w[j]; ph->id[d] = ph->id[j];
      j++;
    }
    ph->n = M;
  }
  /* append */
  for (uint64_t k = 0; k < nnbw; ++k) {
    or_lep_birth *src[2] = {&be[k], &bp[k]};
    or_particles *dst[2] = {e, pos};
    for (int s = 0; s < 2; ++s) {
      or_particles *L = dst[s];
      uint64_t myid = b[0] + 2 * k + s;
      if (!L || L->n >= L->cap) { if (st) st->n_drop++; continue; }
      uint64_t j = L->n++;
      L->x[j] = src[s]->x[0]; L->y[j] = src[s]->x[1]; L->z[j] = src[s]->x[2];
      L->px[j] = src[s]->p[0]; L->py[j] = src[s]->p[1]; L->pz[j] = src[s]->p[2];
      L->s1[j] = src[s]->s[0]; L->s2[j] = src[s]->s[1]; L->s3[j] = src[s]->s[2];
      L->w[j] = src[s]->w; L->id[j] = myid;
    }
  }
  for (uint64_t k = 0; k < nncs; ++k) {
    if (!ph || ph->n >= ph->cap) { if (st) st->n_drop++; continue; }
    uint64_t j = ph->n++;
    ph->x[j] = bg[k].x[0]; ph->y[j] = bg[k].x[1]; ph->z[j] = bg[k].x[2];
    ph->px[j] = bg[k].k[0]; ph->py[j] = bg[k].k[1]; ph->pz[j] = bg[k].k[2];
    ph->s1[j] = bg[k].xi[0]; ph->s2[j] = bg[k].xi[1]; ph->s3[j] = bg[k].xi[2];
    ph->theta[j] = bg[k].th; ph->w[j] = bg[k].w;
    ph->id[j] = k < nncs_e ? b[1] + k : b[2] + (k - nncs_e);
  }
  c->next_id = b[3];
  or_drop_pending(c);
  return 0;
}

int or_step(or_ctx *c, or_particles *e, or_particles *pos, or_particles *ph, const or_fields *f, double t, double dt,
            uint64_t seed, uint32_t step, uint32_t flags, or_stats *st) {
  or_step_decide(c, e, pos, ph, f, t, dt, seed, step, flags, st, NULL);
  return or_step_commit(c, e, pos, ph, NULL, st);
}

/* Ids of one rank's births when R ranks step disjoint parts of one population: the step's
   births are numbered as one sequential pass over the ranks' particles in rank order would
   number them (all pairs, then every e- emission, then every e+ emission), so that the ids
   are unique and gapless across the ranks.  all: R x 3 counts (pairs, e- emissions, e+
   emissions), rank-major; out: the bases of or_step_commit. */
void or_shard_bases(uint64_t next_id, const uint64_t *all, int rank, int world, uint64_t out[4]) {
  uint64_t before[3] = {0, 0, 0}, tot[3] = {0, 0, 0};
  for (int q = 0; q < world; ++q)
    for (int k = 0; k < 3; ++k) {
      tot[k] += all[3 * q + k];
      if (q < rank) before[k] += all[3 * q + k];
    }
  out[0] = next_id + 2 * before[0];
  out[1] = next_id + 2 * tot[0] + before[1];
  out[2] = next_id + 2 * tot[0] + tot[1] + before[2];
  out[3] = next_id + 2 * tot[0] + tot[1] + tot[2];
}
