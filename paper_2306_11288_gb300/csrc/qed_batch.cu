// qed_batch.cu -- batches of independent ensembles: one launch of each step kernel over
// (ensemble, tile) work items, a device-side tile map and clocks so that one captured step
// replays as a CUDA graph, and an autotuner over the launch shape.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "qed_kernels.cuh"

namespace qedk {

// ---- tile map of a batched step --------------------------------------------------------
// one thread per ensemble: its photon tiles, e- tiles, lepton tiles from the live counts
// at the step start, then exclusive prefixes over the ensembles
constexpr int kMapThreads = 1024;

__device__ __forceinline__ unsigned int block_exclusive_scan(unsigned int v, unsigned int* s_w, unsigned int* total) {
  const unsigned int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int c = v;
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
    s_w[lane] = w;
  }
  __syncthreads();
  const unsigned int r = (warp ? s_w[warp - 1] : 0u) + c - v;
  *total = s_w[kMapThreads / 32 - 1];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kMapThreads) k_bmap(const __grid_constant__ StepArgs a) {
  __shared__ unsigned int s_w[kMapThreads / 32];
  const int e = threadIdx.x;
  unsigned int tp = 0, te = 0, tl = 0;
  if (e < a.n_ens) {
    const EnsArgs& E = a.ens[e];
    const DevState* s = E.st;
    const unsigned long long nph = E.sp[2].present ? s->n_live[2] : 0ull;
    const unsigned long long n0 = E.sp[0].present ? s->n_live[0] : 0ull;
    const unsigned long long n1 = E.sp[1].present ? s->n_live[1] : 0ull;
    tp = (unsigned int)((nph + kTile - 1) / kTile);
    te = (unsigned int)((n0 + kTile - 1) / kTile);
    tl = te + (unsigned int)((n1 + kTile - 1) / kTile);
    a.map->lep_e_tiles[e] = te;
  }
  unsigned int tot_p, tot_l;
  const unsigned int ep = block_exclusive_scan(tp, s_w, &tot_p);
  const unsigned int el = block_exclusive_scan(tl, s_w, &tot_l);
  if (e < a.n_ens) {
    a.map->ph_tile0[e] = ep;
    a.map->lep_tile0[e] = el;
  }
  if (e == 0) {
    a.map->ph_tile0[a.n_ens] = tot_p;
    a.map->lep_tile0[a.n_ens] = tot_l;
  }
}

template <typename R, bool kSm>
static void launch_batch_t(const StepArgs& a, const int* nb, cudaStream_t s, cudaStream_t side, cudaEvent_t fork,
                           cudaEvent_t join, bool pdl) {
  k_bmap<<<1, kMapThreads, 0, s>>>(a);
  cudaEventRecord(fork, s);
  cudaStreamWaitEvent(side, fork, 0);
  // the photon pass first: it takes the SMs first and the lepton pass fills in as its blocks
  // retire (lepton first left the photon pass alone at the end: 2.5% slower on 64 ensembles)
  k_photon<R, true, kSm><<<nb[0], kTile, 0, s>>>(a);
  if (a.flags & (QED_F_LL | QED_F_MLL | QED_F_MBMT)) k_lepton<R, true, kSm, true><<<nb[1], kTile, 0, side>>>(a);
  else k_lepton<R, true, kSm><<<nb[1], kTile, 0, side>>>(a);
  cudaEventRecord(join, side);
  cudaStreamWaitEvent(s, join, 0);
  k_scan<R, true><<<2, kScanThreads, 0, s>>>(a, -1);   // both scans, after both passes
  if constexpr (sizeof(R) == 4) {
    if (a.flags & QED_F_MLP) launch_k(k_events_mlp<true>, nb[2] * 2, kMlpRows, s, pdl, a);
    else launch_k(k_events<R, true>, nb[2], kTile, s, pdl, a);
  } else {
    launch_k(k_events<R, true>, nb[2], kTile, s, pdl, a);
  }
}

template <typename R, bool kSm>
static int stream_occupancy(int which) {
  int b = 0;
  if (which == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_photon<R, true, kSm>, kTile, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lepton<R, true, kSm>, kTile, 0);
  return b;
}

}  // namespace qedk

using namespace qedk;

struct qed_batch {
  qed_ctx* ctx;
  int n_ens;
  qed_precision prec;
  double dt;
  uint32_t flags;
  int sms;
  int occ[2][2];                    // [smem_rates][photon, lepton] blocks per SM
  qed_batch_config cfg;
  EnsArgs* d_ens;
  BatchMap* d_map;
  DevState* gst;                    // log cursors, epoch, finished-block counter, status
  unsigned int* tile_cnt[2];
  unsigned int* tile_pre[2];
  void* rec[2];
  unsigned long long rec_cap[2];
  unsigned int* holes;
  cudaStream_t side, cap;
  cudaEvent_t fork, join, t0, t1;
  cudaGraphExec_t exec;
  int graph_ok;                     // exec matches cfg
};

#define BFAIL(code, ...)     \
  do {                       \
    set_error(__VA_ARGS__);  \
    return code;             \
  } while (0)
#define BCK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) BFAIL(QED_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static void batch_free(qed_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->d_ens);
  cudaFree(b->d_map);
  cudaFree(b->gst);
  for (int k = 0; k < 2; ++k) {
    cudaFree(b->tile_cnt[k]);
    cudaFree(b->tile_pre[k]);
    cudaFree(b->rec[k]);
  }
  cudaFree(b->holes);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->t0) cudaEventDestroy(b->t0);
  if (b->t1) cudaEventDestroy(b->t1);
  delete b;
}

static StepArgs batch_args(const qed_batch* b) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.ens = b->d_ens;
  a.map = b->d_map;
  a.n_ens = b->n_ens;
  a.dt = b->dt;
  a.fdt = (float)b->dt;
  a.flags = b->flags;
  a.tables = b->prec == QED_PREC_F64 ? (const void*)b->ctx->tab64 : (const void*)b->ctx->tab32;
  a.mlp = (b->ctx->owner ? b->ctx->owner : b->ctx)->mlp;
  a.st = b->gst;
  for (int k = 0; k < 2; ++k) {
    a.tile_cnt[k] = b->tile_cnt[k];
    a.tile_pre[k] = b->tile_pre[k];
    a.rec[k] = b->rec[k];
    a.rec_cap[k] = b->rec_cap[k];
  }
  a.holes = b->holes;
  return a;
}

static qed_status batch_launch(qed_batch* b, cudaStream_t s, bool pdl) {
  const StepArgs a = batch_args(b);
  const int sm = b->cfg.smem_rates ? 1 : 0;
  int nb[3];
  nb[0] = b->sms * std::max(1, std::min(b->cfg.stream_blocks_per_sm, b->occ[sm][0]));
  nb[1] = b->sms * std::max(1, std::min(b->cfg.stream_blocks_per_sm, b->occ[sm][1]));
  nb[2] = b->sms * b->cfg.event_blocks_per_sm;
  if (b->prec == QED_PREC_F64) {
    if (sm) launch_batch_t<double, true>(a, nb, s, b->side, b->fork, b->join, pdl);
    else launch_batch_t<double, false>(a, nb, s, b->side, b->fork, b->join, pdl);
  } else {
    if (sm) launch_batch_t<float, true>(a, nb, s, b->side, b->fork, b->join, pdl);
    else launch_batch_t<float, false>(a, nb, s, b->side, b->fork, b->join, pdl);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) BFAIL(QED_ERR_CUDA, "batched step launch failed: %s", cudaGetErrorString(e));
  return QED_OK;
}

static unsigned long long tiles_of_cap(const qed_particles* p) { return p ? (p->cap + kTile - 1) / kTile : 0ull; }

extern "C" qed_status qed_batch_create(qed_ctx* ctx, const qed_ensemble* ens, int n_ens, double dt, uint32_t flags,
                                       void* stream, qed_batch** out) {
  if (!out) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: out is NULL");
  *out = nullptr;
  if (!ctx || !ctx->alive) BFAIL(QED_ERR_NOT_INITIALIZED, "qed_batch_create: invalid context");
  if (!ens || n_ens < 1 || n_ens > kMaxEns) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: n_ens must be in [1, %d]", kMaxEns);
  if (!(dt > 0.0) || !std::isfinite(dt)) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: dt must be positive and finite");
  {
    const qed_status rf = check_flag_bits(flags, "qed_batch_create");
    if (rf != QED_OK) return rf;
    if (flags & QED_F_DEPOSIT) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: current deposition is for single steps");
    if (flags & (QED_F_BREMS | QED_F_BH))
      BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: the matter processes are for single steps");
  }
  int prec = -1;
  unsigned long long tp = 1, tl = 1, cap_ph = 0, cap_l = 0;
  for (int i = 0; i < n_ens; ++i) {
    const qed_ensemble& E = ens[i];
    if (!E.ctx || !E.ctx->alive) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: ensemble %d has no valid context", i);
    if (E.ctx->tab64 != ctx->tab64) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: ensemble %d does not share the tables", i);
    if (E.ctx == ctx) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: ensemble %d must have its own context", i);
    for (int j = 0; j < i; ++j)
      if (ens[j].ctx == E.ctx) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: ensembles %d and %d share a context", j, i);
    const qed_particles* all[3] = {E.e, E.pos, E.ph};
    const qed_species want[3] = {QED_ELECTRON, QED_POSITRON, QED_PHOTON};
    for (int k = 0; k < 3; ++k) {
      if (!all[k]) continue;
      if (all[k]->ctx != E.ctx || all[k]->species != want[k])
        BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: ensemble %d set %d is not on its context or has the wrong species", i, k);
      if (prec >= 0 && (int)all[k]->prec != prec) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: mixed precisions");
      prec = (int)all[k]->prec;
    }
    if ((flags & QED_F_NBW) && (!E.e || !E.pos)) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: NBW needs e- and e+ sets");
    const qed_status r = check_fields(&E.fields, "qed_batch_create");
    if (r != QED_OK) return r;
    tp += tiles_of_cap(E.ph);
    tl += tiles_of_cap(E.e) + tiles_of_cap(E.pos);
    cap_ph += E.ph ? E.ph->cap : 0;
    cap_l += (E.e ? E.e->cap : 0) + (E.pos ? E.pos->cap : 0);
  }
  if (tp >= (1ull << 31) || tl >= (1ull << 31)) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_create: batch too large");
  {
    const qed_status rm = check_mlp_flag(ctx, flags, prec < 0 ? QED_PREC_F64 : (qed_precision)prec, "qed_batch_create");
    if (rm != QED_OK) return rm;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  qed_batch* b = new qed_batch();
  memset(b, 0, sizeof(*b));
  b->ctx = ctx;
  b->n_ens = n_ens;
  b->prec = prec < 0 ? QED_PREC_F64 : (qed_precision)prec;
  b->dt = dt;
  b->flags = flags;
  b->cfg.stream_blocks_per_sm = b->prec == QED_PREC_F64 ? 2 : 4;
  b->cfg.event_blocks_per_sm = 2;
  b->cfg.smem_rates = 1;
  cudaError_t e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (b->prec == QED_PREC_F64) {
    b->occ[0][0] = stream_occupancy<double, false>(0); b->occ[0][1] = stream_occupancy<double, false>(1);
    b->occ[1][0] = stream_occupancy<double, true>(0); b->occ[1][1] = stream_occupancy<double, true>(1);
  } else {
    b->occ[0][0] = stream_occupancy<float, false>(0); b->occ[0][1] = stream_occupancy<float, false>(1);
    b->occ[1][0] = stream_occupancy<float, true>(0); b->occ[1][1] = stream_occupancy<float, true>(1);
  }
  // worst case: every photon decays, every lepton emits (one event per particle per step)
  b->rec_cap[0] = cap_ph > 0 ? cap_ph : 1;
  b->rec_cap[1] = cap_l > 0 ? cap_l : 1;
  const size_t rbytes[2] = {nbw_rec_bytes(QED_PREC_F64), ncs_rec_bytes(QED_PREC_F64)};
  const unsigned long long tiles[2] = {tp, tl};
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ens, sizeof(EnsArgs) * n_ens);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_map, sizeof(BatchMap));
  if (e == cudaSuccess) e = cudaMalloc(&b->gst, sizeof(DevState));
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaMalloc(&b->tile_cnt[k], sizeof(unsigned int) * tiles[k]);
    if (e == cudaSuccess) e = cudaMalloc(&b->tile_pre[k], sizeof(unsigned int) * tiles[k]);
    if (e == cudaSuccess) e = cudaMalloc(&b->rec[k], rbytes[k] * b->rec_cap[k]);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->rec[k], 0, rbytes[k] * b->rec_cap[k], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->tile_cnt[k], 0, sizeof(unsigned int) * tiles[k], s);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->holes, sizeof(unsigned int) * b->rec_cap[0]);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t1);
  if (e != cudaSuccess) {
    batch_free(b);
    BFAIL(QED_ERR_CUDA, "qed_batch_create: %s", cudaGetErrorString(e));
  }
  // ensemble arguments, the batch's global state, the ensembles' clocks
  EnsArgs* h = new EnsArgs[n_ens];
  for (int i = 0; i < n_ens; ++i)
    fill_ensemble(h[i], ens[i].e, ens[i].pos, ens[i].ph, &ens[i].fields, ens[i].t0, ens[i].seed, ens[i].step0,
                  ens[i].ctx->st, ens[i].dev_stats);
  e = cudaMemcpyAsync(b->d_ens, h, sizeof(EnsArgs) * n_ens, cudaMemcpyHostToDevice, s);
  DevState g;
  memset(&g, 0, sizeof(g));
  g.epoch = 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->gst, &g, sizeof(g), cudaMemcpyHostToDevice, s);
  struct Clock { double t; unsigned int step; float t_rel, t_mod; };
  static_assert(offsetof(DevState, step) == offsetof(DevState, t) + 8, "clock layout");
  static_assert(offsetof(DevState, t_mod) == offsetof(DevState, t) + 16, "clock layout");
  Clock* clk = new Clock[n_ens];
  for (int i = 0; i < n_ens && e == cudaSuccess; ++i) {
    clk[i].t = ens[i].t0;
    clk[i].step = ens[i].step0;
    step_time_floats(ens[i].t0, ens[i].fields.phi0, &clk[i].t_rel, &clk[i].t_mod);
    e = cudaMemcpyAsync(reinterpret_cast<char*>(ens[i].ctx->st) + offsetof(DevState, t), &clk[i], 20,
                        cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  delete[] h;
  delete[] clk;
  if (e != cudaSuccess) {
    batch_free(b);
    BFAIL(QED_ERR_CUDA, "qed_batch_create: %s", cudaGetErrorString(e));
  }
  *out = b;
  return QED_OK;
}

extern "C" qed_status qed_batch_step(qed_batch* b, void* stream) {
  if (!b) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_step: batch is NULL");
  return batch_launch(b, reinterpret_cast<cudaStream_t>(stream), true);
}

// captures one step on the batch's capture stream (programmatic dependent launches if the
// graph accepts them, else plain ones) and instantiates it
static qed_status batch_capture(qed_batch* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    const bool pdl = attempt == 0;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) BFAIL(QED_ERR_CUDA, "qed_batch_run: begin capture: %s", cudaGetErrorString(e));
    const qed_status r = batch_launch(b, b->cap, pdl);
    e = cudaStreamEndCapture(b->cap, &g);
    if (r != QED_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      continue;
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e == cudaSuccess) {
      b->graph_ok = 1;
      return QED_OK;
    }
    b->exec = nullptr;
    cudaGetLastError();
  }
  BFAIL(QED_ERR_CUDA, "qed_batch_run: the step could not be captured as a graph");
}

extern "C" qed_status qed_batch_run(qed_batch* b, uint32_t nsteps, void* stream) {
  const qedk::NvtxRange nvtx_range("qed_batch_run");
  if (!b) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_run: batch is NULL");
  if (!b->graph_ok) {
    const qed_status r = batch_capture(b);
    if (r != QED_OK) return r;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (uint32_t k = 0; k < nsteps; ++k) BCK(cudaGraphLaunch(b->exec, s));
  return QED_OK;
}

extern "C" qed_status qed_batch_clock(qed_batch* b, int e, double* t, uint32_t* step, void* stream) {
  if (!b || e < 0 || e >= b->n_ens || !t || !step) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_clock: bad arguments");
  EnsArgs h;
  BCK(cudaMemcpy(&h, b->d_ens + e, sizeof(h), cudaMemcpyDeviceToHost));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double tv = 0;
  unsigned int sv = 0;
  BCK(cudaMemcpyAsync(&tv, reinterpret_cast<char*>(h.st) + offsetof(DevState, t), sizeof(tv), cudaMemcpyDeviceToHost, s));
  BCK(cudaMemcpyAsync(&sv, reinterpret_cast<char*>(h.st) + offsetof(DevState, step), sizeof(sv), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  *t = tv;
  *step = sv;
  return QED_OK;
}

extern "C" qed_status qed_batch_get_config(const qed_batch* b, qed_batch_config* cfg) {
  if (!b || !cfg) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_get_config: bad arguments");
  *cfg = b->cfg;
  return QED_OK;
}

extern "C" qed_status qed_batch_set_config(qed_batch* b, const qed_batch_config* cfg) {
  if (!b || !cfg) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_set_config: bad arguments");
  if (cfg->stream_blocks_per_sm < 1 || cfg->stream_blocks_per_sm > 4 || cfg->event_blocks_per_sm < 1 ||
      cfg->event_blocks_per_sm > 8 || (cfg->smem_rates != 0 && cfg->smem_rates != 1))
    BFAIL(QED_ERR_INVALID_ARG, "qed_batch_set_config: values out of range");
  if (memcmp(cfg, &b->cfg, sizeof(*cfg)) != 0) {
    b->cfg = *cfg;
    b->graph_ok = 0;
  }
  return QED_OK;
}

static qed_status batch_processed(qed_batch* b, cudaStream_t s, unsigned long long* v) {
  BCK(cudaMemcpyAsync(v, reinterpret_cast<char*>(b->gst) + offsetof(DevState, processed), sizeof(*v),
                      cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  return QED_OK;
}

extern "C" qed_status qed_batch_tune(qed_batch* b, uint32_t steps_per_candidate, void* stream, qed_batch_config* chosen,
                                     double* rate) {
  if (!b || steps_per_candidate < 1) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_tune: bad arguments");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int sblocks[4] = {1, 2, 3, 4}, eblocks[4] = {1, 2, 4, 8};
  // the candidates (a larger stream count than the occupancy allows repeats a smaller one)
  qed_batch_config cand[32];
  int nc = 0;
  for (int sm = 1; sm >= 0; --sm) {
    const int occ_max = std::max(b->occ[sm][0], b->occ[sm][1]);
    for (int si = 0; si < 4; ++si) {
      if (sblocks[si] > std::max(occ_max, 1)) continue;
      for (int ei = 0; ei < 4; ++ei) cand[nc++] = qed_batch_config{sblocks[si], eblocks[ei], sm};
    }
  }
  // The population grows while the candidates run, and a larger population steps at a higher
  // rate: each candidate is timed twice, once in a forward and once in a backward sweep, and
  // ranked by the mean of its two rates, so that the drift cancels to first order.  A
  // candidate runs as qed_batch_run runs it, replaying its captured graph (the graph may
  // order the two streaming passes otherwise than direct launches do).
  double sum[32] = {0};
  for (int pass = 0; pass < 2; ++pass) {
    for (int k = 0; k < nc; ++k) {
      const int j = pass == 0 ? k : nc - 1 - k;
      qed_status r = qed_batch_set_config(b, &cand[j]);
      if (r == QED_OK) r = qed_batch_run(b, 1, stream);   // capture and settle
      unsigned long long p0 = 0, p1 = 0;
      if (r == QED_OK) r = batch_processed(b, s, &p0);
      if (r != QED_OK) return r;
      BCK(cudaEventRecord(b->t0, s));
      r = qed_batch_run(b, steps_per_candidate, stream);
      if (r != QED_OK) return r;
      BCK(cudaEventRecord(b->t1, s));
      BCK(cudaEventSynchronize(b->t1));
      float ms = 0;
      BCK(cudaEventElapsedTime(&ms, b->t0, b->t1));
      r = batch_processed(b, s, &p1);
      if (r != QED_OK) return r;
      sum[j] += ms > 0 ? (double)(p1 - p0) / (ms * 1e-3) : 0.0;   // particle-steps per second
    }
  }
  double top = -1.0;
  for (int j = 0; j < nc; ++j) top = std::max(top, 0.5 * sum[j]);
  // Rates within 2% of the best count as equal, and among those the most streaming blocks
  // per SM win (then the higher rate): the population keeps growing after the tuning, and a
  // larger population favours the wider grid (64 ensembles at 58M photons: 4 blocks per SM
  // step 5.6% faster than 3, which the tuning, at a third of that population, rated alike).
  qed_batch_config best = b->cfg;
  double best_rate = -1.0;
  for (int j = 0; j < nc; ++j) {
    const double r = 0.5 * sum[j];
    if (r < 0.98 * top) continue;
    if (best_rate < 0.0 || cand[j].stream_blocks_per_sm > best.stream_blocks_per_sm ||
        (cand[j].stream_blocks_per_sm == best.stream_blocks_per_sm && r > best_rate)) {
      best_rate = r;
      best = cand[j];
    }
  }
  const qed_status r = qed_batch_set_config(b, &best);
  if (r != QED_OK) return r;
  if (chosen) *chosen = best;
  if (rate) *rate = best_rate;
  return QED_OK;
}

extern "C" qed_status qed_batch_destroy(qed_batch* b) {
  if (!b) BFAIL(QED_ERR_INVALID_ARG, "qed_batch_destroy: batch is NULL");
  cudaDeviceSynchronize();
  batch_free(b);
  return QED_OK;
}
