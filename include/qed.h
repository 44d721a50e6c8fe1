/*
 * qed.h -- C ABI of the GB300 (sm_103a) spin/polarization-resolved strong-field QED
 * particle step: the per-macroparticle hot path of the particle-in-cell method of
 * Wan et al., "Simulations of spin/polarization-resolved laser-plasma interactions
 * in the nonlinear QED regime" (arXiv:2306.11288).
 *
 * Units (paper Sec. I, last paragraph): time in 1/omega0, length in 1/k0 (the laser
 * wavelength is 2 pi), momentum in m c, energy in m c^2, E and B in m c omega0 / e.
 * The laser wavelength is 1 um, so xi_L = hbar omega0 / m c^2 = 2.42631023867e-6.
 *
 * Conventions shared by every call:
 *   - Every pointer called "device" must point to memory of the current CUDA device;
 *     "host" pointers are ordinary (preferably pinned) host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls marked "async" only enqueue work; calls marked "syncs" block on `stream`.
 *   - Every call returns a qed_status.  Arguments are validated on the host before any
 *     work is enqueued; on a non-OK return nothing has been enqueued and
 *     qed_last_error() holds a message (thread-local).  Nothing throws across the ABI.
 *   - Device-side failures (capacity overflow, a bounded wait that gave up, a table
 *     range clamp) never trap: kernels set bits in a device status word that
 *     qed_read_status() returns.
 *   - The library never frees caller memory.
 */
#ifndef QED_H
#define QED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QED_OK = 0,
  QED_ERR_INVALID_ARG = 1,     /* host-side validation failed                        */
  QED_ERR_CUDA = 2,            /* a CUDA runtime call failed (message says which)    */
  QED_ERR_CAPACITY = 3,        /* births exceeded a particle array's capacity         */
  QED_ERR_NOT_INITIALIZED = 4, /* NULL or destroyed context                          */
  QED_ERR_TIMEOUT = 5,         /* a bounded device wait gave up                       */
  QED_WARN_TABLE_RANGE = 6     /* chi above a table's range was clamped              */
} qed_status;

/* bits of the device status word (qed_read_status) */
#define QED_STATUS_CAPACITY 1u     /* births dropped: a particle array was full             */
#define QED_STATUS_TIMEOUT 2u      /* a bounded device wait gave up                          */
#define QED_STATUS_TABLE_RANGE 4u  /* chi above a table's range was clamped                  */
#define QED_STATUS_LOG_FULL 8u     /* a tile's events were not logged (event log full).  The
                                      logs hold one event per particle of capacity, the most
                                      a step can produce, so this bit marks a library fault */
#define QED_STATUS_SHARD 16u       /* qed_step_end: the gathered counts at this rank's place
                                      differ from the ones qed_step_begin reported (ids of
                                      the ranks would collide)                               */

typedef enum { QED_ELECTRON = 0, QED_POSITRON = 1, QED_PHOTON = 2 } qed_species;

/* Storage precision of a particle set.
 * QED_PREC_F64:   every array is double.
 * QED_PREC_MIXED: positions x, y, z are double; momenta, spins/Stokes, basis angle and
 *                 weights are float; arithmetic is FP32 except the FP64 islands (phase
 *                 and position accumulation, chi under cancellation, the u -> 1 branch). */
typedef enum { QED_PREC_F64 = 0, QED_PREC_MIXED = 1 } qed_precision;

/* process flags of qed_step (paper Sec. IV orders them: Lorentz & T-BMT => VB => NBW => NCS) */
#define QED_F_NCS 1u           /* spin/polarization-resolved nonlinear Compton (Sec. III C)   */
#define QED_F_NBW 2u           /* polarization/spin-resolved nonlinear Breit-Wheeler (III D)  */
#define QED_F_VB 4u            /* vacuum birefringence rotation of photon Stokes (III F)      */
#define QED_F_SPIN 8u          /* T-BMT spin precession (Sec. III B, Eq. bmteqn)             */
#define QED_F_NO_RECOIL 16u    /* test mode: emission changes the spin only, no photon born   */
#define QED_F_DROP_PHOTONS 32u /* emitted photons are not stored (recoil is applied)          */
#define QED_F_MLP 64u          /* NCS photon energy from the learned sampler (mixed path only;
                                  the context or its owner must hold parameters: qed_mlp_*);
                                  events with chi_e outside [1e-3, 10] use the table sampler */
/* Radiative pusher (Sec. III A "Algorithms of the Radiative Pusher", Sec. III B radiative
 * T-BMT): deterministic radiation reaction in place of the NCS Monte Carlo, for the regime
 * where stochasticity does not matter (the paper disables it when NCS is on; combining
 * either with QED_F_NCS is rejected).  Evaluated once per step at the time-centred
 * momentum (p^{n-1/2} + p_L^{n+1/2})/2 of the Boris step and the fields at x^n:
 *   QED_F_LL   : p^{n+1/2} = p_L^{n+1/2} + F_RR dt with the Landau-Lifshitz force of Eq.
 *                eq1-1 (its second and third terms; the field-derivative term is dropped,
 *                the paper notes the last two dominate in ultra-intense fields);
 *   QED_F_MLL  : the same with q(chi) F_RR, q = I_QED/I_C the quantum/classical radiated
 *                power ratio (tabulated from the NCS spectrum; q = 1 below chi = 1e-4);
 *   QED_F_MBMT : half kicks S += dt/2 (dS/dt)_R before and after the T-BMT rotation,
 *                (dS/dt)_R = -P[psi1 S + psi2 (S.beta) beta + psi3 n_B] (Eq. spin1),
 *                n_B = n x a_hat; with QED_F_SPIN this is the paper's M-BMT, alone it is
 *                the radiative term without precession.  S is then a mean polarisation
 *                (|S| <= 1), not a unit vector. */
#define QED_F_LL 128u
#define QED_F_MLL 256u
#define QED_F_MBMT 512u
/* Current deposition (Sec. II C, Esirkepov's charge-conserving scheme with the TSC shape of
 * Sec. II E): every lepton adds the current of its move x^n -> x^{n+1} (charge q w, v_z of
 * p^{n+1/2}) to gJx, gJy, gJz of a QED_FIELD_GRID2D field, so that (rho^{n+1} - rho^n)/dt +
 * div J = 0 on the grid.  Moves of more than one cell per axis (beyond the solver's CFL)
 * are not deposited.  Float atomics: the summation order, and so the last bits of J, vary
 * from run to run.  Single-ensemble steps only (qed_batch_create rejects it). */
#define QED_F_DEPOSIT 1024u
/* Matter (Sec. III E; needs a medium, qed_set_medium): direct Monte Carlo of
 *   QED_F_BREMS: bremsstrahlung of e- and e+ inside the medium, if the lepton had no NCS
 *                event in the step (one event per particle per step): P = 1 - exp(-n sigma(E)
 *                v dt) at the energy of p^{n+1/2} and the position x^n; photon energy
 *                omega = y E from the cumulative cross-section (r sigma(E) = sigma(y, E)),
 *                along p, unpolarised (xi = 0), born at x^{n+1}; the lepton keeps its
 *                direction with energy E - omega (the nucleus takes the momentum balance)
 *                and its spin (the process is not spin-resolved);
 *   QED_F_BH   : Bethe-Heitler pair creation by photons inside the medium that did not
 *                decay by NBW: P = 1 - exp(-n sigma(k) c dt); positron energy x k from the
 *                cumulative cross-section, electron k - x k, both along the photon, born at
 *                its x^n with S = 0 (unpolarised).
 * Cross-sections: Tsai's, with his screening functions for Z >= 5 (see qed_set_medium).
 * Not with the radiative pusher flags; single-ensemble steps only. */
#define QED_F_BREMS 2048u
#define QED_F_BH 4096u

/* Structure-of-arrays view of one species, caller-owned device memory.  Element i of
 * every array describes particle i.  Element types follow qed_precision (above):
 *   x, y, z   : double always
 *   px,py,pz  : lepton momentum p (m c) or photon wave vector k = omega n (m c)
 *   s1,s2,s3  : lepton spin unit vector S (Sec. III B), or photon Stokes parameters
 *               xi1..xi3 (Sec. III C, Stokes parameters paragraph)
 *   theta     : photons only: basis angle; P1 = cos(theta) e1 + sin(theta) e2 with
 *               e1 = unit(y_hat x n) (unit(n x x_hat) within 1e-10 rad of +-y), e2 = n x e1,
 *               and P2 = n x P1.  The Stokes parameters refer to (P1, P2, n).  NULL for leptons.
 *   w         : macro-particle weight (copied to newborns)
 *   id        : uint64 global id (newborns get ids from the context's counter)
 * Arrays must hold `capacity` elements; the first `n` are live. */
typedef struct {
  void *x, *y, *z;
  void *px, *py, *pz;
  void *s1, *s2, *s3;
  void *theta;
  void *w;
  uint64_t *id;
} qed_soa;

/* External field (paper Sec. II D: force deposition onto particles).
 * kind QED_FIELD_UNIFORM : constant E, B.
 * kind QED_FIELD_PLANE   : plane wave moving along -z, phase phi = t + z, sin^2 envelope
 *                          g = a0 sin^2(pi (phi-phi0)/len) on [phi0, phi0+len] (0 outside);
 *                          E = g (cos phi, circular ? sin phi : 0, 0), B = (-z_hat) x E.
 * kind QED_FIELD_GAUSS   : first-order paraxial Gaussian moving along -z, focus z = zf,
 *                          waist w0, Rayleigh length w0^2/2; same envelope in phi; carrier
 *                          phase phi - r^2 zeta/(2(zeta^2+zR^2)) + atan(zeta/zR), zeta = zf - z;
 *                          amplitude w0/w(zeta) exp(-r^2/w^2); longitudinal parts neglected.
 * kind QED_FIELD_GRID2D  : 2D3V Yee grid (z squeezed; paper Sec. II B figure "yeegrid"),
 *                          float arrays [ny][nx] in device memory with Ex(i+1/2,j),
 *                          Ey(i,j+1/2), Ez(i,j), Bx(i,j+1/2), By(i+1/2,j), Bz(i+1/2,j+1/2);
 *                          cell (i, j) at (x0 + i dx, y0 + j dy); gathered with the TSC
 *                          shape of Sec. II E (nodes outside the grid contribute zero). */
typedef enum { QED_FIELD_NONE = 0, QED_FIELD_UNIFORM = 1, QED_FIELD_PLANE = 2,
               QED_FIELD_GAUSS = 3, QED_FIELD_GRID2D = 4 } qed_field_kind;

typedef struct {
  int kind;
  int circular;
  double a0, phi0, len, w0, zf;
  double E[3], B[3];
  const float *gEx, *gEy, *gEz, *gBx, *gBy, *gBz;
  int nx, ny;
  double dx, dy, x0, y0;
  int periodic;              /* grid: 1 = periodic in x and y (gather and deposit wrap),
                                0 = nodes outside the grid are zero                      */
  float *gJx, *gJy, *gJz;    /* grid: current density for QED_F_DEPOSIT, [ny][nx] with
                                Jx(i+1/2,j), Jy(i,j+1/2), Jz(i,j) (the E positions); may
                                be NULL otherwise                                         */
} qed_fields;

/* The 2D3V Yee grid of the field solver (paper Sec. II B, Fig. "yeegrid" (b), z squeezed):
 * nine float arrays [ny][nx] in device memory, caller-owned, with the staggering of
 * QED_FIELD_GRID2D (Ex(i+1/2,j), Ey(i,j+1/2), Ez(i,j), Bx(i,j+1/2), By(i+1/2,j),
 * Bz(i+1/2,j+1/2)) and the current on the E positions.  Normalised units: c = 1, E and B
 * in m c omega/e, J in e n_c c, so that curl B = dE/dt + J and div E = rho (rho in e n_c);
 * a macro-particle of weight w stands for a density w/(dx dy) n_c spread over one cell. */
typedef struct {
  float *Ex, *Ey, *Ez, *Bx, *By, *Bz, *Jx, *Jy, *Jz;
  int nx, ny;
  double dx, dy;
  int periodic;              /* 1 periodic, 0 neighbours outside the grid are zero */
} qed_grid2d;

/* Per-step event counters accumulated on the device (add-only). */
typedef struct {
  uint64_t n_ncs[2];     /* photon emissions by e-, e+                         */
  uint64_t n_nbw;        /* pairs created                                      */
  uint64_t n_range;      /* chi clamped at a table's upper edge                */
  uint64_t n_drop;       /* births dropped for lack of capacity                */
  uint64_t n_steps;      /* steps accumulated                                  */
  uint64_t n_processed;  /* particle-steps: live e-, e+, photons at each step start */
  uint64_t n_coarse;     /* decisions whose probability W dt (NCS) or T dt (NBW) exceeded
                            0.1: the step allows one event per particle, which is a coarse
                            description of such a step -- a smaller dt is advisable      */
  uint64_t n_brems[2];   /* bremsstrahlung events of e-, e+ (QED_F_BREMS)         */
  uint64_t n_bh;         /* Bethe-Heitler pairs (QED_F_BH)                        */
} qed_step_stats;

typedef struct qed_ctx qed_ctx;             /* tables, id counter, scratch, status   */
typedef struct qed_particles qed_particles; /* non-owning SoA view + device count      */

/* Build the QED lookup tables on the current device (FP64 quadrature on the GPU) and
 * return a context.  Tables: scaled K_1/3, K_2/3, IntK_1/3 (Eqs. F0-F3, G0-G3); the
 * u-integrated spin-resolved NCS rate of Eq. Wspin2; inverse CDFs of the photon energy
 * fraction for spin projections +-1; the spin-summed NBW rate (Eq. BW summed over both
 * spins) and inverse CDFs of the positron energy fraction for xi3' = +-1; the VB
 * functions M_par, M_perp of Sec. III F.  Syncs `stream`.  *out receives a context
 * that the caller releases with qed_destroy.  Errors: QED_ERR_INVALID_ARG (out NULL),
 * QED_ERR_CUDA. */
qed_status qed_init_tables(qed_ctx **out, void *stream);

/* Release a context and its device memory (tables, scratch).  Syncs the device. */
qed_status qed_destroy(qed_ctx *ctx);

/* Wrap caller-owned device arrays as one species (paper Sec. IV: ParticleList).
 * `buffers` pointers are copied; the arrays must outlive the returned object.  All
 * particle sets stepped together must share one precision.  `n` <= `capacity` <= 2^32 - 256.
 * The live count lives in the context (one set per species per context).  Grows the
 * context's step scratch (event logs, per-tile counts) to the capacity.
 * Syncs `stream`.  Errors: QED_ERR_INVALID_ARG (NULL array, n > capacity, photon
 * without theta), QED_ERR_CUDA. */
qed_status particles_create(qed_ctx *ctx, qed_species species, const qed_soa *buffers,
                            uint64_t n, uint64_t capacity, qed_precision prec, void *stream,
                            qed_particles **out);

/* Live count (device word) into *n.  Syncs `stream`. */
qed_status particles_count(const qed_particles *p, uint64_t *n, void *stream);

/* Overwrite the live count (e.g. after refilling the arrays).  Async. */
qed_status particles_set_count(qed_particles *p, uint64_t n, void *stream);

/* Release the wrapper and its count word (not the caller's arrays).  Syncs the device. */
qed_status particles_destroy(qed_particles *p);

/* Id counter of newborn particles (ids of primaries are the caller's).  set: async;
 * get: syncs `stream`. */
qed_status qed_set_next_id(qed_ctx *ctx, uint64_t next_id, void *stream);
qed_status qed_get_next_id(qed_ctx *ctx, uint64_t *next_id, void *stream);

/* One time step of every live particle (async, graph-capturable: no host sync, no
 * allocation).  The lepton pass runs on a side stream of the context, forked from and
 * joined back into `stream` by events, so all of the step's work is ordered after earlier
 * work on `stream` and before later work on it.  Order (paper Sec. IV and the leapfrog of
 * Sec. II F):
 *   photons: gather E, B at x^n, t; rotate Stokes into the local pair frame (Eq.
 *     rotation); VB phase (Eq. rotation2) if QED_F_VB; NBW decision and pair sampling
 *     (Sec. III D) if QED_F_NBW; survivors move x += dt n; decayed photons are removed
 *     (stable); pairs are born at the photon's x^n.
 *   leptons (e- then e+): Boris push (Eqs. boris1-6), T-BMT rotation (Eqs. bmt-boris1-4)
 *     if QED_F_SPIN, x^{n+1} = x^n + dt p^{n+1/2}/gamma; chi_e; NCS decision from the
 *     spin-resolved total rate (Eq. Wspin2 integrated over u); no-emission spin update
 *     and collapse, or emission: photon energy, recoil, spin collapse along the SQA of
 *     Eq. F0, photon pure state from Eqs. F1-F3; photons are born at x^{n+1}.
 *   newborns are appended after the survivors and are first advanced at the next step.
 * Ids of newborns: next_id + ... in the order NBW pairs (photon order; e- then e+), then
 * NCS photons (e- order, then e+ order).  Random numbers: Philox4x32-10 with key = seed
 * and counter = (id_lo, id_hi, step, stream index).
 * e, pos, ph may be NULL (an absent species); all given sets share one precision.
 * dev_stats (device memory, optional) accumulates counters.
 *   with QED_F_LL / QED_F_MLL / QED_F_MBMT the radiative pusher (see the flags) acts
 *     between the Boris push and the position update, and NCS is off.
 * Errors: QED_ERR_INVALID_ARG (dt <= 0 or not finite, precision mismatch, unknown
 * field kind, NULL grid arrays, NBW without lepton arrays, unknown flag bits, the
 * radiative pusher together with QED_F_NCS, QED_F_LL with QED_F_MLL),
 * QED_ERR_NOT_INITIALIZED, QED_ERR_CUDA (launch failure). */
qed_status qed_step(qed_ctx *ctx, qed_particles *e, qed_particles *pos, qed_particles *ph,
                    const qed_fields *f, double t, double dt, uint64_t seed, uint32_t step,
                    uint32_t flags, qed_step_stats *dev_stats, void *stream);

/* A step of one part of a population that several ranks (one process per GPU) step
 * together, each its own particles (Sec. IV: particles are independent given the fields).
 * The only exchange is the births' ids, so that they stay unique and gapless across the
 * ranks: a step numbers its births as one sequential pass over all ranks' particles in rank
 * order would (every rank's pairs, then every e- emission, then every e+ emission; within a
 * rank, qed_step's order).  Every rank keeps the same id counter.
 *   qed_step_begin: the step up to its event kernel (both streaming passes and the scans;
 *     same arguments and validation as qed_step); writes this rank's three birth counts
 *     (pairs, e- emissions, e+ emissions; uint64) to dev_counts (device memory) on stream.
 *   Then the caller gathers every rank's dev_counts into dev_all (world x 3, rank-major;
 *     an all-gather of 24 bytes per rank, e.g. ncclAllGather on the same stream).
 *   qed_step_end: the births with ids offset by the ranks before this one, and the rest of
 *     the step; the counter advances by all ranks' births.  Sets QED_STATUS_SHARD if
 *     dev_all at this rank's place is not what qed_step_begin wrote.
 * With world = 1 the two calls equal one qed_step.  Between them the context, the particle
 * sets and dev_counts must stay as they are; no other step on the context.
 * Errors: as qed_step; QED_ERR_INVALID_ARG (qed_step_end without qed_step_begin, NULL
 * dev_counts / dev_all, rank outside [0, world), a second qed_step_begin before the end,
 * per-kernel timing on). */
qed_status qed_step_begin(qed_ctx *ctx, qed_particles *e, qed_particles *pos, qed_particles *ph,
                          const qed_fields *f, double t, double dt, uint64_t seed, uint32_t step,
                          uint32_t flags, qed_step_stats *dev_stats, uint64_t *dev_counts, void *stream);
qed_status qed_step_end(qed_ctx *ctx, const uint64_t *dev_all, int rank, int world, void *stream);

/* Matter for QED_F_BREMS and QED_F_BH (paper Sec. III E, high-energy bremsstrahlung and
 * the Bethe-Heitler pair creation that "follows a similar process"): atoms of charge Z at
 * n atoms per normalised volume (1/k0^3; for a solid of density rho in g/cm^3 and molar
 * mass A: n = rho N_A / A (1e-4 / 2 pi)^3), filling the slab lo <= x[axis] < hi (normalised
 * units; axis 0, 1, 2 = x, y, z); photons below k_min (m c^2) are not produced.
 * Cross-sections (Tsai, Rev. Mod. Phys. 46, 815 (1974), the paper's reference):
 *   brems  dsigma/dy = alpha r0^2 / y [(4/3 - 4/3 y + y^2) A + (2/3)(1 - y) B], y = omega/E,
 *   pairs  dsigma/dx = alpha r0^2 [(1 - 4/3 x(1-x)) A - (2/3) x(1-x) B], x = E+/k,
 *   A = Z^2 (phi1 - 4/3 ln Z - 4 f) + Z (psi1 - 8/3 ln Z), B = Z^2 (phi1 - phi2) + Z (psi1 - psi2)
 * with Tsai's screening functions phi1,2, psi1,2 for Thomas-Fermi atoms (valid for Z >= 5)
 * and the Coulomb correction f(Z); where the fits leave their range (no screening near the
 * end points, low energies) a negative brace counts as zero.  Builds the cumulative tables
 * on the device (FP64; 256 energies from 1 to 1e6 MeV x 512 nodes uniform in the logit
 * of the energy fraction) and keeps them on the context; syncs `stream`.  m NULL removes
 * the medium.  Errors: QED_ERR_INVALID_ARG (Z outside [5, 100], n or k_min not positive,
 * axis outside 0..2, lo >= hi), QED_ERR_NOT_INITIALIZED, QED_ERR_CUDA. */
typedef struct {
  int Z;
  double n;
  double k_min;
  int axis;
  double lo, hi;
} qed_medium;
qed_status qed_set_medium(qed_ctx *ctx, const qed_medium *m, void *stream);
/* Diagnostics: the medium's FP64 tables to host memory (syncs): brems rows then pair rows,
 * [2][256 energies][512 nodes], each row the cumulative cross-section (units alpha r0^2)
 * from the low end of the energy fraction.  *len receives 2 * 256 * 512; host may be NULL
 * to query it.  Errors: QED_ERR_INVALID_ARG (no medium set, cap too small). */
qed_status qed_copy_medium_table(qed_ctx *ctx, double *host, uint64_t cap, uint64_t *len, void *stream);

/* Field solver (Sec. II B): one half of the Yee leapfrog on a 2D3V grid (async).
 *   which = QED_FDTD_B: B -= dt curl E   (Faraday);
 *   which = QED_FDTD_E: E += dt (curl B - J) (Ampere), and J is then set to zero, ready
 *                       for the next step's deposition.
 * Only the curl equations are solved: with the charge-conserving deposition Gauss's law
 * is kept (Sec. II B).  The PIC loop of Sec. II F around qed_step, with E^n and B^{n-1/2}
 * stored: FDTD_B(dt/2); qed_step(... | QED_F_DEPOSIT) gathers E^n, B^n and deposits
 * J^{n+1/2}; FDTD_B(dt/2); FDTD_E(dt).  The explicit scheme needs dt below the 2D Courant
 * limit 1/sqrt(1/dx^2 + 1/dy^2).  Errors: QED_ERR_INVALID_ARG (NULL arrays, nx or ny < 2,
 * ny > 65535, dx, dy or dt not positive and finite, unknown which), QED_ERR_CUDA. */
#define QED_FDTD_B 0
#define QED_FDTD_E 1
qed_status qed_fdtd_advance(const qed_grid2d *g, int which, double dt, void *stream);

/* Cell sort of one particle set on a 2D grid (async; no host synchronisation): the live
 * particles are reordered by 32x32-cell tile of `grid` (a QED_FIELD_GRID2D descriptor; only
 * its geometry is used) and, inside a tile, by cell (row-major); particles outside a
 * bounded grid go last; a periodic grid wraps positions.  The cell of x is
 * floor((x - x0) * (1/dx)), each operation rounded in double (likewise y).  Stable: particles of one cell keep
 * their order, so the result is deterministic.  Every array of the set is permuted (the
 * live part).  A PIC code sorts periodically: the gather and the deposition of a warp then
 * touch a few cache lines (Sec. II D, E: field and current interpolation on the grid).
 * Scratch (48 B per element of capacity plus 512 KB) is allocated on the context on first
 * use and kept.  Errors: QED_ERR_INVALID_ARG (not a grid, set of another context, capacity
 * >= 2^32, grid too large for 32-bit keys), QED_ERR_NOT_INITIALIZED, QED_ERR_CUDA. */
qed_status qed_sort_cells(qed_ctx *ctx, qed_particles *set, const qed_fields *grid, void *stream);

/* End-to-end form of qed_step for callers whose particles live in host memory: copies
 * the live part of each given host SoA (same layout and precision as the device set,
 * counts n_host[3] for e-, e+, photons) into the device sets, runs one qed_step, and
 * copies the device sets back (capacity elements are available in the host arrays;
 * n_host is updated with the new counts).  host_soa[k] may be NULL for an absent
 * species.  Syncs `stream`. */
qed_status qed_step_host(qed_ctx *ctx, qed_particles *e, qed_particles *pos, qed_particles *ph,
                         const qed_soa *host_e, const qed_soa *host_pos, const qed_soa *host_ph,
                         uint64_t n_host[3], const qed_fields *f, double t, double dt,
                         uint64_t seed, uint32_t step, uint32_t flags, void *stream);

/* qed_step for callers that cannot allocate device memory when they step -- code that
 * runs while its stream is captured into a CUDA graph, or an application whose device
 * memory is all owned by its own allocator.  The paper has no counterpart of this call.
 * It runs exactly the kernels of qed_step, but keeps their per-step scratch (per-tile event
 * counts and prefixes, the event logs sized for one event per particle, the list of
 * decayed photon slots) in one file-scope device array of the library (about 17.8 MiB,
 * held by every process that loads the library on every device it uses) instead of the
 * context's buffers, and calls no cudaMalloc or cudaFree.  Limit: every given particle
 * set must have capacity <= 65536; larger sets are rejected with QED_ERR_INVALID_ARG (use
 * qed_step).  A call outside stream capture looks the array's address up
 * (cudaGetSymbolAddress) with the device current and keeps it; a call inside a capture
 * uses the kept address, so make the first call on a device (and the first after a
 * cudaDeviceReset) outside any capture -- otherwise QED_ERR_INVALID_ARG.  Every call, on every context of the
 * process, shares the array and leaves its contents behind; a step reads only entries it
 * has written, so nothing needs clearing.  Calls whose work overlaps on the GPU (other
 * streams, other threads, other contexts) race on the array: order them on one stream.
 * The context, its tables and the particle sets are created as for qed_step.
 * Arguments, order of processes, ids and errors are those of qed_step.  Async. */
qed_status qed_step_static(qed_ctx *ctx, qed_particles *e, qed_particles *pos, qed_particles *ph,
                           const qed_fields *f, double t, double dt, uint64_t seed, uint32_t step,
                           uint32_t flags, qed_step_stats *dev_stats, void *stream);

/* Device status word (QED_STATUS_* bits) accumulated since the last clear; syncs
 * `stream`.  clear != 0 resets it. */
qed_status qed_read_status(qed_ctx *ctx, uint32_t *status, int clear, void *stream);

/* Diagnostics: per-kernel timing.  While enabled, qed_step runs all its kernels on `stream`
 * one after the other (no side stream, no programmatic dependent launches), records CUDA
 * events around the photon streaming kernel, the lepton streaming kernel and the event
 * kernels, and waits for them, adding the elapsed milliseconds to three accumulators (so
 * every step syncs and is slower than an untimed one).  qed_get_timing returns and clears
 * them with the number of steps timed.  Off by default. */
qed_status qed_set_timing(qed_ctx *ctx, int enable);
qed_status qed_get_timing(qed_ctx *ctx, double ms[3], uint64_t *steps);

/* Diagnostics: copy one FP64 lookup table of the context to host memory (syncs).
 * which: 0 scaled K13, K23, IntK13 values then their d/dln x, [2][3][1024] on ln x in
 *          [ln 1e-3, ln 1e5];
 *        1 NCS A(chi)/chi then B(chi)/chi, [2][512] on ln chi in [ln 1e-4, ln 1e3];
 *        2 NCS inverse CDF: ln u then d(ln u)/dt, [2][2 spin projections +1,-1][256 chi]
 *          [512 t], t = logit(level) in [-38, 38];
 *        3 NBW T0 then T3, each times exp(8/(3 chi_g)), [2][256] on ln chi_g in
 *          [ln 1e-2, ln 1e3];
 *        4 NBW half inverse CDF: ln delta then d(ln delta)/dt, [2][2 xi3' = +1,-1][256 chi_g]
 *          [256 t], t = ln(level of the half distribution) in [-38, 0];
 *        5 VB M_par then M_perp, [2][1024] on ln chi_g in [ln 1e-3, ln 1e3];
 *        6 radiative pusher q(chi), psi1/chi^3, psi2/chi^3, psi3/chi^3, [4][512] on the
 *          grid of 1;
 *        7 the mixed path's float interval cubics of the 1-D tables, returned as doubles:
 *          VB M_par - M_perp [1021][4], NBW T0, T3 [253][2][4], NCS A/chi, B/chi
 *          [509][2][4], radiative pusher (the four tables of 6) [509][4][4]; row r holds
 *          the 4-point Lagrange interpolant of node interval i = r + 1 as c0..c3 with
 *          p(f) = c0 + f (c1 + f (c2 + f c3)), f = X - i (X in grid units).
 * *len receives the element count; host may be NULL to query it; otherwise cap must be
 * >= the count.  Errors: QED_ERR_INVALID_ARG (bad which, cap too small). */
qed_status qed_copy_table(qed_ctx *ctx, int which, double *host, uint64_t cap, uint64_t *len, void *stream);

/* Diagnostics: the step's random-number generator, Philox4x32-10 (Salmon et al., SC'11,
 * the counter-based generator every Monte Carlo decision of the step draws from), run on
 * the device for n counters under one 64-bit key.
 * ctr: device memory, n x 4 words (counter words 0..3 of each block); key: key word 0 in
 * the low 32 bits, key word 1 in the high 32 bits; out: device memory, n x 8 words --
 * words 0..3 of each block from the form that derives the ten round keys inside the kernel
 * (batched launches), words 4..7 from the form that takes them precomputed on the host as
 * kernel parameters (single-ensemble launches).  The two halves must agree.  Async on
 * `stream`; the caller owns both buffers.  Errors: QED_ERR_INVALID_ARG (NULL buffer with
 * n > 0), QED_ERR_CUDA (launch failure). */
qed_status qed_philox_blocks(const uint32_t *ctr, uint64_t key, uint32_t *out, uint64_t n, void *stream);

/* ---- End-of-run observables (paper Sec. IV: post-processing of the photon polarization,
 * Figs. of spectra, mean spin and pair yield) ------------------------------------------
 * qed_diag histograms one particle set on the device.
 *   kind QED_DIAG_SPECTRUM: nx bins uniform in ln(energy) over [lo_x, hi_x) (0 < lo_x <
 *     hi_x); energy = |k| for photons, gamma = sqrt(1 + p^2) for leptons; ny must be 1.
 *   kind QED_DIAG_DETECTOR: nx * ny cells uniform in the particle position (x, y) over
 *     [lo_x, hi_x) x [lo_y, hi_y) (the detection plane of the paper's VB post-processing).
 * Per bin the call accumulates {sum w, sum w o1, sum w o2, sum w o3, count}, where o is the
 * spin vector (Sx, Sy, Sz) for leptons and, for photons, the Stokes parameters rotated by
 * Eq. (rotation) from the photon's stored basis to the detection basis (d1, d2 = n x d1),
 * d1 = unit(ref - (ref . n) n) with ref = spec->ref (x if ref is zero; the canonical basis
 * vector e1 of n if ref is parallel to n).
 * dev_out (device, caller-owned, FP64) receives 5 * (nx * ny) bin values (bin-major: bin
 * i at [5 i .. 5 i + 4], bin index ix + nx * iy), then the same five values over every
 * particle of the set, then sum w below and sum w above the range (x axis; for the
 * detector, outside in either coordinate counts as "above"): 5 * (nx * ny + 1) + 2
 * doubles.  Sums are FP64: per-block partials, then a fixed-order compensated (Neumaier)
 * sum over blocks.  Async; no host sync unless the context's diagnostic scratch must
 * grow.  Errors: QED_ERR_INVALID_ARG (NULL pointers, nx * ny outside [1, 1024], bad
 * ranges, ny != 1 for a spectrum). */
typedef enum { QED_DIAG_SPECTRUM = 0, QED_DIAG_DETECTOR = 1 } qed_diag_kind;
typedef struct {
  int kind;
  int nx, ny;
  double lo_x, hi_x, lo_y, hi_y;
  double ref[3];
} qed_diag_spec;
qed_status qed_diag(qed_ctx *ctx, const qed_particles *set, const qed_diag_spec *spec, double *dev_out,
                    void *stream);

/* ---- Batches of independent ensembles (many collisions stepped together) ---------------
 * The paper's method applies per macroparticle; a batch steps many independent ensembles
 * (each a set of e-, e+, photons in its own external field, with its own clock, step
 * counter, RNG key and id counter) with one launch of each step kernel over all of them
 * (work items = (ensemble, tile)).  Each ensemble's results are those qed_step would give
 * it alone.  The paper has no counterpart of batching: it is an execution scheme. */

/* A context that uses `parent`'s tables (built once) with its own device state: live
 * counts, id counter, step scratch.  An ensemble's particle sets are created on such a
 * context.  `parent` must own its tables and outlive the shared context.  Syncs nothing.
 * Errors: QED_ERR_NOT_INITIALIZED (parent), QED_ERR_INVALID_ARG, QED_ERR_CUDA. */
qed_status qed_ctx_share(qed_ctx *parent, void *stream, qed_ctx **out);

typedef struct {
  qed_ctx *ctx;                 /* the ensemble's context (made by qed_ctx_share) */
  qed_particles *e, *pos, *ph;  /* its sets, created on ctx (any may be NULL) */
  qed_fields fields;            /* its external field (copied; grid arrays must stay valid) */
  double t0;                    /* its time at the batch's first step */
  uint32_t step0;               /* its step number at the first step (RNG counter) */
  uint64_t seed;                /* its RNG key */
  qed_step_stats *dev_stats;    /* optional device statistics, accumulated */
} qed_ensemble;

/* launch shape of a batched step (see qed_batch_tune) */
typedef struct {
  int stream_blocks_per_sm;     /* streaming passes: 1..4 (capped by occupancy) */
  int event_blocks_per_sm;      /* event kernels: 1..8 */
  int smem_rates;               /* 1: 1-D rate tables staged in shared memory; 0: read via L1/L2 */
} qed_batch_config;

typedef struct qed_batch qed_batch;

/* Creates a batch of n_ens (1..1024) ensembles on the context `ctx` (its tables; the
 * ensembles' contexts must share them).  All sets must have one precision.  Every step
 * advances each ensemble's clock by dt and its step number by one, on the device.
 * Allocates the batch's scratch (sized from the sets' capacities) and copies the clocks to
 * the ensembles' device state (syncs `stream`).  Errors: QED_ERR_INVALID_ARG (sizes,
 * mixed precisions, a set not on its ensemble's context, contexts not sharing ctx's
 * tables, flags), QED_ERR_CUDA. */
qed_status qed_batch_create(qed_ctx *ctx, const qed_ensemble *ens, int n_ens, double dt, uint32_t flags,
                            void *stream, qed_batch **out);

/* One step of every ensemble (async, graph-capturable, no allocation): a tile-map kernel,
 * then the kernels of qed_step with (ensemble, tile) work items, the lepton pass on the
 * batch's side stream. */
qed_status qed_batch_step(qed_batch *b, void *stream);

/* nsteps steps by replaying one captured step as a CUDA graph (captured on first use and
 * again after a configuration change).  Async. */
qed_status qed_batch_run(qed_batch *b, uint32_t nsteps, void *stream);

/* Reads ensemble e's clock (syncs).  Errors: QED_ERR_INVALID_ARG (e out of range). */
qed_status qed_batch_clock(qed_batch *b, int e, double *t, uint32_t *step, void *stream);

qed_status qed_batch_get_config(const qed_batch *b, qed_batch_config *cfg);
/* Errors: QED_ERR_INVALID_ARG (values out of range). */
qed_status qed_batch_set_config(qed_batch *b, const qed_batch_config *cfg);

/* Autotuner: runs steps_per_candidate real steps of the batch under each candidate launch
 * shape (streaming blocks per SM x event blocks per SM x rate-table placement) as
 * qed_batch_run runs them (a captured graph, replayed), times them with CUDA events, and
 * keeps the one with the most particle-steps per second.  The
 * population grows while the candidates run, so every candidate is timed twice, in a
 * forward and in a backward sweep, and ranked by the mean of its two rates; rates within
 * 2% of the best count as equal, and among those the shape with the most streaming blocks
 * per SM is kept (the population keeps growing, and larger populations favour the wider
 * grid).  The steps
 * (2 x (steps_per_candidate + 1) per candidate) advance the simulation; the results do not
 * depend on the launch shape.  Syncs.  *rate (optional) receives the chosen shape's mean
 * particle-steps per second.  Errors: QED_ERR_INVALID_ARG, QED_ERR_CUDA. */
qed_status qed_batch_tune(qed_batch *b, uint32_t steps_per_candidate, void *stream, qed_batch_config *chosen,
                          double *rate);

qed_status qed_batch_destroy(qed_batch *b);

/* ---- Learned photon-energy sampler of the NCS events -----------------------------------
 * A 3 -> 64 -> 64 -> 1 GELU network maps (ln chi_e, s = S.zeta, one uniform r) to ln u,
 * u = omega/(gamma - omega), in place of the two-component inverse-CDF table lookup (the
 * spin mixture of Eq. Wspin2, inverted as one monotone map of r).  Its 64 x 64 layer runs on
 * the tensor cores in BF16 with FP32 accumulation; the rest in FP32.  The paper has no
 * counterpart: this is an alternative sampler, judged against the table sampler.
 * Parameters live on the context that owns the tables (a shared context uses its owner's).
 * Parameter vector (4481 floats): w1[64][3], b1[64], w2[64][64], b2[64], w3[64], b3. */

/* Trains on n_samples samples produced by the table sampler itself (ln chi_e uniform in
 * [ln 1e-3, ln 10], s uniform in [-1, 1], r uniform -- for 1/16 of the samples
 * logit(r) uniform in [-38, 38] to cover the tails; target its mixture inverse CDF from the
 * FP32 tables), in batches of `batch`, with Adam and a cosine learning rate, from an
 * initialisation seeded by `seed`.  The number of Adam steps (n_samples / batch) sets the
 * fit: 1e8 samples in batches of 1024 (about 1e5 steps, ~10 s on a GB300) reach a median ln u
 * error of ~1e-3 against the table sampler.  Syncs.  Errors: QED_ERR_INVALID_ARG (64 <=
 * batch <= 2^22, batch <= n_samples), QED_ERR_CUDA. */
qed_status qed_mlp_train(qed_ctx *ctx, uint64_t n_samples, uint32_t batch, uint64_t seed, void *stream);
/* Copy the parameter vector in or out (host, 4481 floats; syncs). */
qed_status qed_mlp_set_params(qed_ctx *ctx, const float *host, void *stream);
qed_status qed_mlp_get_params(qed_ctx *ctx, float *host, void *stream);
/* ln u of the learned sampler (tensor cores) and of the table sampler's mixture inverse for
 * n device rows (ln chi_e, s, r) -> dev_out[n] (async).  Errors: QED_ERR_NOT_INITIALIZED (no
 * parameters, for qed_mlp_eval), QED_ERR_INVALID_ARG. */
qed_status qed_mlp_eval(qed_ctx *ctx, const float *dev_in, float *dev_out, uint64_t n, void *stream);
qed_status qed_mlp_target(qed_ctx *ctx, const float *dev_in, float *dev_out, uint64_t n, void *stream);

/* Message of the last failing call on this thread ("" if none). */
const char *qed_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
