/*
 * qed_oracle.h -- plain, slow, FP64 CPU oracle of the spin/polarization-resolved
 * strong-field QED particle step of Wan et al., "Simulations of spin/polarization-
 * resolved laser-plasma interactions in the nonlinear QED regime" (arXiv:2306.11288).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this code: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg use it.  It shares no code with the CUDA library.
 *
 * Units (paper Sec. I, normalisation paragraph): t in 1/omega0, x in 1/k0,
 * p in m c, E and B in m c omega0 / e, energies in m c^2.
 *
 * Parity status per function is stated in oracle/qed_oracle.c's header comment.
 */
#ifndef QED_ORACLE_H
#define QED_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* --- process flags (same meaning as the library's QED_F_* flags) ----------- */
#define OR_F_NCS        1u   /* nonlinear Compton (Sec. III C)                 */
#define OR_F_NBW        2u   /* nonlinear Breit-Wheeler (Sec. III D)            */
#define OR_F_VB         4u   /* vacuum birefringence (Sec. III F)               */
#define OR_F_SPIN       8u   /* T-BMT precession (Sec. III B, Eq. bmteqn)       */
#define OR_F_NO_RECOIL 16u   /* test mode: emission leaves p unchanged, no photon */
#define OR_F_DROP_PHOTONS 32u /* emitted photons are not stored (recoil kept)  */
#define OR_F_LL       128u   /* classical Landau-Lifshitz radiation reaction (Eq. eq1-1) */
#define OR_F_MLL      256u   /* quantum-corrected LL: q(chi) F_RR,classical (Sec. III A) */
#define OR_F_MBMT     512u   /* radiative T-BMT (Eq. spin1); needs OR_F_SPIN        */
#define OR_F_DEPOSIT 1024u   /* leptons deposit their current (Esirkepov, Sec. II C)  */
#define OR_F_BREMS   2048u   /* bremsstrahlung of leptons in matter (Sec. III E)       */
#define OR_F_BH      4096u   /* Bethe-Heitler pair creation by photons in matter (III E) */

/* --- particle arrays (structure of arrays, caller-owned) -------------------- */
typedef struct {
  double *x, *y, *z;       /* position                                          */
  double *px, *py, *pz;    /* lepton momentum, or photon k = omega * n          */
  double *s1, *s2, *s3;    /* lepton spin unit vector, or photon Stokes xi1..3  */
  double *theta;           /* photons: basis angle (NULL for leptons)           */
  double *w;               /* macro weight                                      */
  uint64_t *id;            /* global id                                         */
  uint64_t n;              /* live count (updated by or_step)                   */
  uint64_t cap;            /* capacity                                          */
} or_particles;

/* --- external field descriptor ---------------------------------------------- */
enum { OR_FIELD_NONE = 0, OR_FIELD_UNIFORM = 1, OR_FIELD_PLANE = 2,
       OR_FIELD_GAUSS = 3, OR_FIELD_GRID2D = 4 };
typedef struct {
  int kind;
  int circular;            /* 0: linear (E along x), 1: circular              */
  double a0;               /* peak amplitude per component                     */
  double phi0, len;        /* sin^2 envelope over phi = t + z in [phi0, phi0+len] */
  double w0;               /* Gaussian waist (normalised, k0 w0)               */
  double zf;               /* focal plane z                                    */
  double E[3], B[3];       /* uniform fields                                   */
  /* 2D3V Yee grid (x,y), fields constant along z */
  const float *gEx, *gEy, *gEz, *gBx, *gBy, *gBz;
  int nx, ny;
  double dx, dy, x0, y0;
  int periodic;            /* grid: 1 periodic in x and y, 0 nodes outside are zero */
  double *gJx, *gJy, *gJz; /* grid current (OR_F_DEPOSIT adds to it), [ny][nx] with
                              Jx(i+1/2,j) Jy(i,j+1/2) Jz(i,j)                       */
} or_fields;

/* --- 2D3V Yee grid of the field solver (Sec. II B), double, [ny][nx] ----------
 * Ex(i+1/2,j) Ey(i,j+1/2) Ez(i,j) Bx(i,j+1/2) By(i+1/2,j) Bz(i+1/2,j+1/2), currents on
 * the E positions; node (i,j) at (x0 + i dx, y0 + j dy).  Normalised units: c = 1,
 * E, B in m c omega/e, rho in e n_c, J in e n_c c, so that div E = rho and
 * curl B = dE/dt + J.  A macro-particle of weight w carries density w/(dx dy) n_c. */
typedef struct {
  double *Ex, *Ey, *Ez, *Bx, *By, *Bz, *Jx, *Jy, *Jz;
  int nx, ny;
  double dx, dy;
  int periodic;
} or_grid;

typedef struct {
  uint64_t n_ncs[2];       /* emissions by e-, e+                             */
  uint64_t n_nbw;          /* pair creations                                   */
  uint64_t n_range;        /* chi clamped at a table's upper edge              */
  uint64_t n_drop;         /* births dropped for lack of capacity              */
  uint64_t n_near;         /* decisions within the near-tie tolerance (logged) */
  uint64_t n_coarse;       /* decisions with probability W dt or T dt above 0.1 */
  uint64_t n_brems[2];     /* bremsstrahlung events of e-, e+                   */
  uint64_t n_bh;           /* Bethe-Heitler pairs                               */
} or_stats;

/* Matter for bremsstrahlung and Bethe-Heitler pairs (Sec. III E): atoms of charge Z
 * (Tsai's screening functions are for Z >= 5) at n atoms per normalised volume (k0^-3),
 * filling the slab lo <= x[axis] < hi; photons below k_min (m c^2) are not produced. */
typedef struct {
  int Z;
  double n;
  double k_min;
  int axis;
  double lo, hi;
} or_medium;

/* kinds of the discrete decisions of a step (near-tie log) */
enum { OR_D_NCS = 0,          /* emission: r < W dt (Sec. III C)                     */
       OR_D_NCS_COLLAPSE = 1, /* no-emission spin sign: r < (1 + |S_bar|)/2          */
       OR_D_NCS_COMP = 2,     /* spin component of the energy mixture (Eq. Wspin2)   */
       OR_D_NCS_SPIN = 3,     /* final spin sign along the SQA of Eq. F0             */
       OR_D_NCS_STOKES = 4,   /* photon pure-state sign: r < (1 + |F|/F0)/2          */
       OR_D_NBW = 5,          /* pair creation: r < T dt (Sec. III D)                */
       OR_D_NBW_COMP = 6,     /* xi3' component of the energy mixture                */
       OR_D_NBW_SPIN = 7,     /* one of the three cumulative thresholds of the 4-way pick */
       OR_D_BREMS = 8,        /* bremsstrahlung: r < 1 - exp(-n sigma v dt) (Sec. III E) */
       OR_D_BH = 9 };         /* Bethe-Heitler pair: r < 1 - exp(-n sigma c dt)        */

typedef struct or_ctx or_ctx;

/* tables of Sec. III C-F; built once (seconds) */
or_ctx *or_ctx_create(void);
void or_ctx_destroy(or_ctx *c);
void or_set_next_id(or_ctx *c, uint64_t id);
uint64_t or_get_next_id(const or_ctx *c);
/* Near-tie log: every decision "r < thr" of or_step with |r - thr| < tol thr is recorded
 * as (id, step, kind, margin = |r - thr|/thr); tol defaults to 1e-6.  or_near_log copies up
 * to cap entries (in the order the decisions were taken) and returns the number logged
 * since the last or_set_next_id (which clears the log). */
void or_set_near_tol(or_ctx *c, double tol);
/* Threads of the particle loops of or_step (OpenMP; ignored with OR_F_DEPOSIT, whose
 * current sums into one grid).  Results are the same for any count.  Returns the count
 * in effect (1 when the oracle was built without OpenMP). */
int or_set_threads(or_ctx *c, int n);
uint64_t or_near_log(or_ctx *c, uint64_t *ids, uint32_t *steps, uint32_t *kinds, double *margins, uint64_t cap);

int or_step(or_ctx *c, or_particles *e, or_particles *pos, or_particles *ph,
            const or_fields *f, double t, double dt, uint64_t seed, uint32_t step,
            uint32_t flags, or_stats *st);
/* or_step in two parts: every decision of the step (the particles are updated in place,
 * the births held); counts = (pairs, e- emissions, e+ emissions) when non-NULL.  Then the
 * births with the ids bases[0] + 2k + s (pair k, s = 0 e-, 1 e+), bases[1] + k (the k-th
 * e- emission), bases[2] + k (e+), and the counter at bases[3]; NULL bases number them from
 * the counter in that order (or_step).  Commit returns -1 without a decided step. */
int or_step_decide(or_ctx *c, or_particles *e, or_particles *pos, or_particles *ph,
                   const or_fields *f, double t, double dt, uint64_t seed, uint32_t step,
                   uint32_t flags, or_stats *st, uint64_t counts[3]);
int or_step_commit(or_ctx *c, or_particles *e, or_particles *pos, or_particles *ph,
                   const uint64_t *bases, or_stats *st);
/* the bases of rank `rank` of `world` ranks stepping disjoint parts of one population:
 * its births are numbered as one pass over all ranks' particles in rank order would number
 * them; all = world x 3 counts of or_step_decide, rank-major */
void or_shard_bases(uint64_t next_id, const uint64_t *all, int rank, int world, uint64_t out[4]);

/* Yee leapfrog halves (Sec. II B): B -= dt curl E;  E += dt (curl B - J) */
void or_fdtd_b(const or_grid *g, double dt);
void or_fdtd_e(const or_grid *g, double dt);
/* TSC charge density of n particles (charge*weight qw) on the nodes: rho += ... */
void or_charge_tsc(const or_grid *g, double x0, double y0, const double *x, const double *y,
                   const double *qw, uint64_t n, double *rho);

/* --- pieces exposed for the oracle's own pins ------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_uniforms(uint64_t seed, uint64_t id, uint32_t step, uint32_t ctr, double u[2]);
void or_besselk_scaled(double x, double out[3]);   /* e^x{K13, K23, IntK13}(x) */
void or_ktable(const or_ctx *c, double x, double out[3]);
void or_ncs_rates(const or_ctx *c, double chi, double out[2]);      /* A, B     */
double or_ncs_invcdf(const or_ctx *c, int comp, double chi, double t); /* ln u */
void or_nbw_rates(const or_ctx *c, double chig, double out[2]);     /* T0, T3   */
double or_nbw_invcdf(const or_ctx *c, int comp, double chig, double t); /* ln d */
void or_vb_m(const or_ctx *c, double chig, double out[2]);          /* M_par, M_perp */
/* matter (Sec. III E): set the medium (builds its tables; NULL removes it) */
void or_set_medium(or_ctx *c, const or_medium *m);
/* Tsai's screening functions phi1, phi2 (gamma), psi1, psi2 (eps); Coulomb correction */
void or_screening(double g, double e, double out[4]);
double or_coulomb_f(int Z);
/* braces of the cross-sections: dsigma/dy = alpha r0^2 D_b / y (y = omega/E, E total
   lepton energy), dsigma/dx = alpha r0^2 D_p (x = E+/k) */
double or_brems_D(int Z, double E, double y);
double or_pair_D(int Z, double k, double x);
/* total cross-section (units alpha r0^2; which 0 brems above k_min, 1 pairs) at energy E
   by the tables, and the sampled y or x for a uniform r */
double or_medium_sigma(const or_ctx *c, int which, double E);
double or_medium_sample(const or_ctx *c, int which, double E, double r);
/* radiative pusher functions at chi (Sec. III A, B): out = {q, psi1, psi2, psi3} */
void or_rr_funcs(const or_ctx *c, double chi, double out[4]);
double or_scorer_gi_prime(double y);
void or_field(const or_fields *f, double x, double y, double z, double t,
              double E[3], double B[3]);
/* F0..F3 of Eqs. F0-F3 at (u, chi) for spins Si, Sf in frame (n, a) */
void or_ncs_F(const or_ctx *c, double u, double chi, const double n[3],
              const double a[3], const double Si[3], const double Sf[3], double F[4]);
/* G0..G3 of Eqs. G0-G3 (common W0/2 dropped, K's scaled by e^rho) */
void or_nbw_G(const or_ctx *c, double delta, double omega, double chig,
              const double ap[3], const double bp[3], const double vp[3],
              const double Sp[3], const double Sm[3], double G[4]);
/* raw table access for pins: which = 0 K, 1 ncs rate, 2 ncs inv, 3 nbw rate,
   4 nbw inv, 5 vb, 6 radiative pusher (q, psi1/chi^3, psi2/chi^3, psi3/chi^3),
   7 medium: brems cumulative [256][512] then pair cumulative [256][512] */
const double *or_table(const or_ctx *c, int which, uint64_t *len);

#ifdef __cplusplus
}
#endif
#endif
