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

struct StepArgs {
  SpeciesArgs sp[3];                 // e-, e+, photon
  qed_fields f;
  double t, dt;
  unsigned long long seed;
  unsigned int step, flags;
  const void* tables;                // double* or float* depending on precision
  DevState* st;
  unsigned long long* look[2];       // decoupled look-back words: photon, lepton tiles
  unsigned long long look_cap[2];    // words available
  qed_step_stats* user_stats;
};

// launches one step (photon kernel, lepton kernel); prec selects the instantiation.
// ev (optional): three events recorded before, between and after the kernels.
qed_status launch_step(const StepArgs& a, qed_precision prec, int nblk_ph, int nblk_lep, cudaStream_t s,
                       cudaEvent_t* ev);
// occupancy-derived persistent grid sizes
qed_status step_grid_sizes(qed_precision prec, int* nblk_ph, int* nblk_lep);

constexpr int kTile = 256;   // particles per tile (= threads per block, one particle each)

}  // namespace qedk

struct qed_ctx {
  int device;
  double* tab64;
  float* tab32;
  qedk::DevState* st;
  unsigned long long* look[2];
  unsigned long long look_cap[2];
  int nblk[2][2];   // [precision][photon, lepton]
  int alive;
  int timing;
  cudaEvent_t tev[3];
  double tms[2];
  unsigned long long tsteps;
};

struct qed_particles {
  qed_ctx* ctx;
  qed_species species;
  qed_precision prec;
  qed_soa soa;
  unsigned long long cap;
};
