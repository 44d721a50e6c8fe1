// qed_internal.h -- host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/qed.h"

namespace qedk {

struct DevState;

// thread-local error message (qed_last_error)
void set_error(const char* fmt, ...);

// builds the FP64 tables into d64 (kTableLen doubles) and the float copy into d32
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
};

struct StepArgs {
  SpeciesArgs sp[3];                 // e-, e+, photon
  qed_fields f;
  double t, dt;
  double inv_len;                    // 1 / envelope length
  FloatConsts ff;
  unsigned long long seed;
  unsigned int step, flags;
  const void* tables;                // double* or float* depending on precision
  DevState* st;
  unsigned int* tile_cnt[2];         // events per tile: photon tiles, lepton tiles
  unsigned int* tile_pre[2];         // their exclusive prefixes
  void* rec[2];                      // event logs: NBW decays, NCS emissions
  unsigned long long rec_cap[2];
  unsigned int* holes;               // ranked slots of decayed photons
  qed_step_stats* user_stats;
};

// side stream and events of one step.  side == nullptr runs everything on the caller's
// stream.  tev (optional, timing): [0] step start, [1] end of the photon pass, [3] step
// end (caller's stream); [4], [5] around the lepton pass (on the stream that runs it).
struct StreamSet {
  cudaStream_t side;
  cudaEvent_t fork, join;
  cudaEvent_t* tev;
};

// launches one step; prec selects the instantiation; nblk = grid sizes (photon, lepton,
// events)
qed_status launch_step(const StepArgs& a, qed_precision prec, const int* nblk, cudaStream_t s, const StreamSet& ss);
// occupancy-derived persistent grid sizes
qed_status step_grid_sizes(qed_precision prec, int* nblk);
size_t nbw_rec_bytes(qed_precision p);
size_t ncs_rec_bytes(qed_precision p);

constexpr int kTile = 256;   // particles per tile (= threads per block, one particle each)

}  // namespace qedk

struct qed_ctx {
  int device;
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
};

struct qed_particles {
  qed_ctx* ctx;
  qed_species species;
  qed_precision prec;
  qed_soa soa;
  unsigned long long cap;
};
