// qed_internal.h -- host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>

#include "../../include/qed.h"

namespace qedk {

struct DevState;

// thread-local error message (qed_last_error)
void set_error(const char* fmt, ...);

// NVTX range over a host entry point (visible in Nsight timelines; inert without a tool)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// builds the FP64 tables into d64 (kTableLen doubles) and the float copy with the
// mixed path's interval cubics into d32 (kTab32Len floats)
qed_status build_tables(double* d64, float* d32, cudaStream_t st);

// per-launch parameters of the step kernels (one struct, passed by value)
struct SpeciesArgs {
  double *x, *y, *z;
  void *px, *py, *pz, *s1, *s2, *s3, *theta, *w;
  uint64_t* id;
  unsigned long long cap;
  int present;
};

// float copies of per-step constants for the mixed path (no FP64 arithmetic in kernels)
struct FloatConsts {
  float dt, inv_len, t_rel, t_mod, a0, w0, zf, zr, inv_zr, inv_w02;
  // grid: 1/dx = gix + gix_lo and 1/dy (float splits); x0/dx = gox_i + gox + gox_lo and
  // y0/dy likewise (integer part and float split of the fraction)
  float gix, gix_lo, giy, giy_lo, gox, gox_lo, goy, goy_lo;
  int gox_i, goy_i;
};

// the arguments of one ensemble (a set of e-, e+, photons in one field)
struct EnsArgs {
  SpeciesArgs sp[3];                 // e-, e+, photon
  qed_fields f;
  double t;                          // time (single-ensemble launches; batched: DevState::t)
  double inv_len;                    // 1 / envelope length
  FloatConsts ff;                    // float constants; t_rel, t_mod only for single launches
  unsigned long long seed;
  unsigned int rk[20];               // Philox key schedule of seed (single-ensemble launches)
  unsigned int step;                 // step number (single launches; batched: DevState::step)
  DevState* st;                      // the ensemble's counts, id counter, per-step totals
  qed_step_stats* user_stats;
};

// Batched steps: where each ensemble's tiles and events start.  Rebuilt on the device at
// the start of every batched step from the live counts (k_bmap) and by the scans.
constexpr int kMaxEns = 1024;
struct BatchMap {
  unsigned int ph_tile0[kMaxEns + 1];     // first photon tile of each ensemble; [n] = total
  unsigned int lep_tile0[kMaxEns + 1];    // first lepton tile (its e- tiles, then its e+ tiles)
  unsigned int lep_e_tiles[kMaxEns];      // e- tiles of each ensemble
  unsigned int ev_base[2][kMaxEns + 1];   // first rank of each ensemble's decays / emissions
};

// per-launch parameters of the step kernels (one struct, passed by value)
struct StepArgs {
  EnsArgs e0;                        // single-ensemble launches
  const EnsArgs* ens;                // batched launches: n_ens entries in device memory
  BatchMap* map;
  int n_ens;
  double dt;
  float fdt;
  unsigned int flags;
  const void* tables;                // double* or float* depending on precision
  const void* mlp;                   // learned sampler parameters (QED_F_MLP)
  DevState* st;                      // log cursors, epoch, finished-block counter, status
  unsigned int* tile_cnt[2];         // events per tile: photon tiles, lepton tiles
  unsigned int* tile_pre[2];         // their exclusive prefixes
  void* rec[2];                      // event logs: NBW decays, NCS emissions
  unsigned long long rec_cap[2];
  unsigned int* holes;               // ranked slots of decayed photons
  // matter (QED_F_BREMS, QED_F_BH): cumulative tables (brems rows, then pair rows), the
  // row totals as floats, n alpha r0^2, the slab, k_min
  const double* med_c;
  const float* med_tot;
  double med_nar2, med_lo, med_hi, med_kmin;
  int med_axis;
  // sharded steps (qed_step_begin / qed_step_end): this rank's birth counts out, every
  // rank's counts in (world x 3, rank-major)
  unsigned long long* shard_counts;
  const unsigned long long* shard_all;
  int shard_rank, shard_world;
};

// side stream and events of one step.  side == nullptr runs everything on the caller's
// stream.  tev (optional, timing): [0] step start, [1] end of the photon pass, [3] step
// end (caller's stream); [4], [5] around the lepton pass (on the stream that runs it).
struct StreamSet {
  cudaStream_t side;
  cudaEvent_t fork, join;
  cudaEvent_t* tev;
};

// launches one step of one ensemble (a.e0); prec selects the instantiation; nblk = grid
// sizes (photon, lepton, events)
// which part of a step launch_step runs: all of it, or the two halves of a sharded step
// (up to the scans and the rank's birth counts / the id offsets and the event kernel)
enum StepPart { kStepWhole = 0, kStepBegin = 1, kStepEnd = 2 };
qed_status launch_step(const StepArgs& a, qed_precision prec, const int* nblk, cudaStream_t s, const StreamSet& ss,
                       StepPart part = kStepWhole);
// fills one ensemble's arguments (sets may be NULL; t, step: the ensemble's clock)
void fill_ensemble(EnsArgs& E, const qed_particles* e, const qed_particles* pos, const qed_particles* ph,
                   const qed_fields* f, double t, uint64_t seed, uint32_t step, DevState* st,
                   qed_step_stats* stats);
void step_time_floats(double t, double phi0, float* t_rel, float* t_mod);
// the ten Philox4x32-10 round keys of seed: rk[2r] = lo + r W0, rk[2r+1] = hi + r W1
void philox_key_schedule(uint64_t seed, unsigned int rk[20]);
// the generator check of qed_philox_blocks (arguments validated by the caller)
cudaError_t launch_philox_blocks(const uint32_t* ctr, uint64_t key, uint32_t* out, uint64_t n, cudaStream_t s);
// host validation of a field descriptor (message prefixed by who)
qed_status check_fields(const qed_fields* f, const char* who);
qed_status check_deposit(uint32_t flags, const qed_fields* f, const char* who);
}  // namespace qedk
struct qed_ctx;
namespace qedk {
// QED_F_MLP needs the mixed path and trained (or set) sampler parameters
// every flag bit the step kernels know; validation of flag combinations
constexpr uint32_t kAllFlags = 8191u;
qed_status check_flag_bits(uint32_t flags, const char* who);
qed_status check_mlp_flag(const qed_ctx* c, uint32_t flags, qed_precision prec, const char* who);
// the step's medium arguments from the context (nothing if it has no medium)
void set_medium_args(StepArgs& a, const qed_ctx* c);
// occupancy-derived persistent grid sizes
qed_status step_grid_sizes(qed_precision prec, int* nblk);
size_t nbw_rec_bytes(qed_precision p);
size_t ncs_rec_bytes(qed_precision p);

constexpr int kTile = 256;   // particles per tile (= threads per block, one particle each)

}  // namespace qedk

struct qed_ctx {
  int device;
  int shared;                         // tables belong to another context (qed_ctx_share)
  qed_ctx* owner;                     // that context (NULL for an owner)
  void* mlp;                          // learned sampler parameters (owner only)
  int mlp_ready;
  double* tab64;
  float* tab32;
  qedk::DevState* st;
  // step scratch, sized for the largest particle sets created on this context
  unsigned long long cap_seen[3];     // e-, e+, photon capacities
  unsigned int* tile_cnt[2];
  unsigned int* tile_pre[2];
  unsigned long long tile_cap[2];
  void* rec[2];
  unsigned long long rec_cap[2];
  unsigned int* holes;
  int nblk[2][3];   // [precision][photon, lepton, events]
  int alive;
  cudaStream_t side;                  // lepton pass runs here, overlapping the photon chain
  cudaEvent_t fork, join;
  int timing;
  cudaEvent_t tev[6];
  double tms[3];
  unsigned long long tsteps;
  void* diag_buf;                     // per-block partial histograms of qed_diag
  size_t diag_bytes;
  void* sort_buf;                     // qed_sort_cells scratch (keys, indices, one array)
  size_t sort_bytes;
  qedk::StepArgs pend;                // a sharded step between qed_step_begin and qed_step_end
  qed_precision pend_prec;
  int pending;
  void* med_buf;                      // medium tables (qed_set_medium)
  qed_medium med;
  int has_medium;
};

struct qed_particles {
  qed_ctx* ctx;
  qed_species species;
  qed_precision prec;
  qed_soa soa;
  unsigned long long cap;
};
