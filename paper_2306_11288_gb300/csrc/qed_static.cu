// qed_static.cu -- qed_step_static: one step for callers that cannot allocate device
// memory when they step (for example code that runs while a stream is being captured into
// a CUDA graph, or a host application whose device memory is all owned by its own pool).
// qed_step keeps its per-step scratch (per-tile event counts and prefixes, the two event
// logs, the ranked list of decayed photon slots) in buffers that particles_create sizes
// with cudaMalloc; this entry point keeps that scratch in one file-scope __device__ array
// instead and allocates nothing.  The price is a fixed limit: at most kStaticMaxCap
// particles of capacity per species.  The paper has no counterpart of this entry point.
#include <cmath>
#include <cstring>
#include <mutex>

#include "qed_common.cuh"
#include "qed_internal.h"

namespace qedk {

constexpr unsigned long long kStaticMaxCap = 65536;   // capacity limit per species
constexpr unsigned long long kStTilesPh = (kStaticMaxCap + kTile - 1) / kTile + 1;
constexpr unsigned long long kStTilesLep = 2 * ((kStaticMaxCap + kTile - 1) / kTile) + 1;
// event logs for the worst case: every photon decays, every e- and e+ emits
constexpr unsigned long long kStRecNbw = kStaticMaxCap;
constexpr unsigned long long kStRecNcs = 2 * kStaticMaxCap;
constexpr size_t kAlign = 256;
constexpr size_t rnd(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }
// layout of the array (byte offsets); logs are sized for the FP64 record layout
constexpr size_t kSoCntPh = 0;
constexpr size_t kSoPrePh = kSoCntPh + rnd(4 * kStTilesPh);
constexpr size_t kSoCntLep = kSoPrePh + rnd(4 * kStTilesPh);
constexpr size_t kSoPreLep = kSoCntLep + rnd(4 * kStTilesLep);
constexpr size_t kSoHoles = kSoPreLep + rnd(4 * kStTilesLep);
constexpr size_t kSoLogNbw = kSoHoles + rnd(4 * kStRecNbw);
constexpr size_t kNbwRecMax = 152, kNcsRecMax = 64;   // bytes per record, bounds checked at run time
constexpr size_t kSoLogNcs = kSoLogNbw + rnd(kNbwRecMax * kStRecNbw);
constexpr size_t kStaticBytes = kSoLogNcs + rnd(kNcsRecMax * kStRecNcs);   // about 17.8 MiB

// One array per process and device, shared by every call and every context.
static __device__ __align__(256) unsigned char g_step_scratch[kStaticBytes];

// Host code cannot use g_step_scratch's name as a device address: the address is looked
// up with the device current.  Every call that is not being captured looks it up again (a
// device reset or another context may have moved it) and caches it per device; a call
// inside a stream capture uses the cache, which a first call outside capture has filled.
static std::mutex g_addr_mu;
static void* g_addr[256];

static qed_status scratch_address(cudaStream_t stream, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("qed_step_static: cudaGetDevice: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  if (dev < 0 || dev >= 256) {
    set_error("qed_step_static: device ordinal %d out of range", dev);
    return QED_ERR_CUDA;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) {
    set_error("qed_step_static: cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_step_scratch);
    if (e != cudaSuccess || !p) {
      set_error("qed_step_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return QED_ERR_CUDA;
    }
    g_addr[dev] = p;
  } else if (!g_addr[dev]) {
    set_error("qed_step_static: the first call on a device must be made outside stream capture");
    return QED_ERR_INVALID_ARG;
  }
  *out = g_addr[dev];
  return QED_OK;
}


}  // namespace qedk

using namespace qedk;

extern "C" qed_status qed_step_static(qed_ctx* c, qed_particles* e, qed_particles* pos, qed_particles* ph,
                                      const qed_fields* f, double t, double dt, uint64_t seed, uint32_t step,
                                      uint32_t flags, qed_step_stats* dev_stats, void* stream) {
  if (!c || !c->alive) {
    set_error("qed_step_static: invalid context");
    return QED_ERR_NOT_INITIALIZED;
  }
  if (c->pending) {
    set_error("qed_step_static: a sharded step is between qed_step_begin and qed_step_end");
    return QED_ERR_INVALID_ARG;
  }
  if (!f) {
    set_error("qed_step_static: fields is NULL");
    return QED_ERR_INVALID_ARG;
  }
  if (!(dt > 0.0) || !std::isfinite(dt)) {
    set_error("qed_step_static: dt must be positive and finite");
    return QED_ERR_INVALID_ARG;
  }
  {
    const qed_status rf = check_flag_bits(flags, "qed_step_static");
    if (rf != QED_OK) return rf;
  }
  const qed_particles* all[3] = {e, pos, ph};
  const qed_species want[3] = {QED_ELECTRON, QED_POSITRON, QED_PHOTON};
  int prec = -1;
  for (int k = 0; k < 3; ++k) {
    if (!all[k]) continue;
    if (all[k]->ctx != c || all[k]->species != want[k]) {
      set_error("qed_step_static: particle set %d does not belong here", k);
      return QED_ERR_INVALID_ARG;
    }
    if (prec >= 0 && (int)all[k]->prec != prec) {
      set_error("qed_step_static: mixed precisions");
      return QED_ERR_INVALID_ARG;
    }
    prec = (int)all[k]->prec;
    if (all[k]->cap > kStaticMaxCap) {
      set_error("qed_step_static: capacity %llu of particle set %d exceeds the limit of %llu per species "
                "(use qed_step for larger sets)", (unsigned long long)all[k]->cap, k, kStaticMaxCap);
      return QED_ERR_INVALID_ARG;
    }
  }
  if ((flags & (QED_F_NBW | QED_F_BH)) && (!e || !pos)) {
    set_error("qed_step_static: NBW and Bethe-Heitler pairs need e- and e+ sets");
    return QED_ERR_INVALID_ARG;
  }
  if ((flags & (QED_F_BREMS | QED_F_BH)) && !c->has_medium) {
    set_error("qed_step_static: QED_F_BREMS / QED_F_BH need a medium (qed_set_medium)");
    return QED_ERR_INVALID_ARG;
  }
  {
    qed_status rf = check_fields(f, "qed_step_static");
    if (rf == QED_OK) rf = check_deposit(flags, f, "qed_step_static");
    if (rf != QED_OK) return rf;
  }
  const qed_precision pr = prec < 0 ? QED_PREC_F64 : (qed_precision)prec;
  {
    const qed_status rm = check_mlp_flag(c, flags, pr, "qed_step_static");
    if (rm != QED_OK) return rm;
  }
  if (nbw_rec_bytes(pr) > kNbwRecMax || ncs_rec_bytes(pr) > kNcsRecMax) {
    set_error("qed_step_static: event record larger than the static layout assumes");
    return QED_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  qed_status r = scratch_address(reinterpret_cast<cudaStream_t>(stream), &base);
  if (r != QED_OK) return r;
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // Nothing is cleared: the array keeps the previous call's contents, and a step reads
  // only entries it has written itself -- every tile's count (the streaming passes write
  // one per tile, events or not), the first `cursor` log records (a log holds the worst
  // case, so every reserved record is written) and the ranked decay slots.
  StepArgs a;
  memset(&a, 0, sizeof(a));
  fill_ensemble(a.e0, e, pos, ph, f, t, seed, step, c->st, dev_stats);
  a.dt = dt;
  a.fdt = (float)dt;
  a.flags = flags;
  a.tables = pr == QED_PREC_F64 ? (const void*)c->tab64 : (const void*)c->tab32;
  a.mlp = (c->owner ? c->owner : c)->mlp;
  a.st = c->st;
  a.tile_cnt[0] = reinterpret_cast<unsigned int*>(b + kSoCntPh);
  a.tile_pre[0] = reinterpret_cast<unsigned int*>(b + kSoPrePh);
  a.tile_cnt[1] = reinterpret_cast<unsigned int*>(b + kSoCntLep);
  a.tile_pre[1] = reinterpret_cast<unsigned int*>(b + kSoPreLep);
  a.holes = reinterpret_cast<unsigned int*>(b + kSoHoles);
  set_medium_args(a, c);
  a.rec[0] = b + kSoLogNbw;
  a.rec[1] = b + kSoLogNcs;
  a.rec_cap[0] = kStRecNbw;
  a.rec_cap[1] = kStRecNcs;
  const int pi = pr == QED_PREC_F64 ? 0 : 1;
  const StreamSet ss{c->side, c->fork, c->join, nullptr};
  return launch_step(a, pr, c->nblk[pi], s, ss);
}
