// qed_api.cu -- the C ABI declared in include/qed.h: argument validation, context and
// particle-set bookkeeping, and the host-buffer (end-to-end) form of the step.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "qed_common.cuh"
#include "qed_internal.h"

namespace qedk {
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
}  // namespace qedk

using namespace qedk;

#define FAIL(code, ...)       \
  do {                        \
    set_error(__VA_ARGS__);   \
    return code;              \
  } while (0)

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) FAIL(QED_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" const char* qed_last_error(void) { return g_err; }

extern "C" qed_status qed_init_tables(qed_ctx** out, void* stream) {
  const qedk::NvtxRange nvtx_range("qed_init_tables");
  if (!out) FAIL(QED_ERR_INVALID_ARG, "qed_init_tables: out is NULL");
  *out = nullptr;
  g_err[0] = 0;
  qed_ctx* c = (qed_ctx*)calloc(1, sizeof(qed_ctx));
  if (!c) FAIL(QED_ERR_INVALID_ARG, "qed_init_tables: host allocation failed");
  CK(cudaGetDevice(&c->device));
  cudaError_t e = cudaMalloc(&c->tab64, sizeof(double) * kTableLen);
  if (e == cudaSuccess) e = cudaMalloc(&c->tab32, sizeof(float) * kTab32Len);
  if (e == cudaSuccess) e = cudaMalloc(&c->st, sizeof(DevState));
  if (e != cudaSuccess) {
    cudaFree(c->tab64); cudaFree(c->tab32); cudaFree(c->st); free(c);
    FAIL(QED_ERR_CUDA, "qed_init_tables: cudaMalloc: %s", cudaGetErrorString(e));
  }
  DevState h;
  memset(&h, 0, sizeof(h));
  h.epoch = 1;
  e = cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, S(stream));
  if (e != cudaSuccess) {
    cudaFree(c->tab64); cudaFree(c->tab32); cudaFree(c->st); free(c);
    FAIL(QED_ERR_CUDA, "qed_init_tables: %s", cudaGetErrorString(e));
  }
  qed_status r = build_tables(c->tab64, c->tab32, S(stream));
  if (r == QED_OK) r = step_grid_sizes(QED_PREC_F64, c->nblk[0]);
  if (r == QED_OK) r = step_grid_sizes(QED_PREC_MIXED, c->nblk[1]);
  if (r != QED_OK) {
    cudaFree(c->tab64); cudaFree(c->tab32); cudaFree(c->st); free(c);
    return r;
  }
  if (r == QED_OK) {
    e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaFree(c->tab64); cudaFree(c->tab32); cudaFree(c->st); free(c);
      FAIL(QED_ERR_CUDA, "qed_init_tables: side stream: %s", cudaGetErrorString(e));
    }
  }
  c->alive = 1;
  *out = c;
  return QED_OK;
}

extern "C" qed_status qed_ctx_share(qed_ctx* parent, void* stream, qed_ctx** out) {
  if (!out) FAIL(QED_ERR_INVALID_ARG, "qed_ctx_share: out is NULL");
  *out = nullptr;
  if (!parent || !parent->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_ctx_share: invalid parent context");
  if (parent->shared) FAIL(QED_ERR_INVALID_ARG, "qed_ctx_share: the parent must own its tables");
  qed_ctx* c = (qed_ctx*)calloc(1, sizeof(qed_ctx));
  if (!c) FAIL(QED_ERR_INVALID_ARG, "qed_ctx_share: host allocation failed");
  c->device = parent->device;
  c->tab64 = parent->tab64;
  c->tab32 = parent->tab32;
  c->shared = 1;
  c->owner = parent;
  memcpy(c->nblk, parent->nblk, sizeof(c->nblk));
  cudaError_t e = cudaMalloc(&c->st, sizeof(DevState));
  DevState h;
  memset(&h, 0, sizeof(h));
  h.epoch = 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, S(stream));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaFree(c->st);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork) cudaEventDestroy(c->fork);
    free(c);
    FAIL(QED_ERR_CUDA, "qed_ctx_share: %s", cudaGetErrorString(e));
  }
  c->alive = 1;
  *out = c;
  return QED_OK;
}

extern "C" qed_status qed_destroy(qed_ctx* c) {
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_destroy: invalid context");
  cudaDeviceSynchronize();
  if (!c->shared) {
    cudaFree(c->tab64);
    cudaFree(c->tab32);
    cudaFree(c->mlp);
  }
  cudaFree(c->st);
  for (int k = 0; k < 2; ++k) {
    cudaFree(c->tile_cnt[k]); cudaFree(c->tile_pre[k]); cudaFree(c->rec[k]);
  }
  cudaFree(c->holes);
  for (int k = 0; k < 6; ++k)
    if (c->tev[k]) cudaEventDestroy(c->tev[k]);
  if (c->diag_buf) cudaFree(c->diag_buf);
  if (c->sort_buf) cudaFree(c->sort_buf);
  if (c->med_buf) cudaFree(c->med_buf);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  if (c->side) cudaStreamDestroy(c->side);
  c->alive = 0;
  free(c);
  return QED_OK;
}

static unsigned long long tiles_of(unsigned long long n) { return (n + kTile - 1) / kTile; }

// (Re)sizes the step scratch for the largest capacities seen on this context:
// per-tile event counts and prefixes, the two event logs (the FP64 record size) and the
// ranked hole list.  The logs are sized for the worst case -- every live photon decays and
// every live lepton emits in one step (at most one event per particle per step) -- so a
// step never drops an event.
static qed_status grow_scratch(qed_ctx* c, cudaStream_t s) {
  const unsigned long long tp = tiles_of(c->cap_seen[2]) + 1;
  const unsigned long long tl = tiles_of(c->cap_seen[0]) + tiles_of(c->cap_seen[1]) + 1;
  const unsigned long long rn = c->cap_seen[2] > 0 ? c->cap_seen[2] : 1;
  const unsigned long long rl = c->cap_seen[0] + c->cap_seen[1] > 0 ? c->cap_seen[0] + c->cap_seen[1] : 1;
  const unsigned long long want_t[2] = {tp, tl}, want_r[2] = {rn, rl};
  const size_t rbytes[2] = {nbw_rec_bytes(QED_PREC_F64), ncs_rec_bytes(QED_PREC_F64)};
  bool sync_done = false;
  for (int k = 0; k < 2; ++k) {
    if (want_t[k] > c->tile_cap[k]) {
      if (!sync_done) { CK(cudaStreamSynchronize(s)); sync_done = true; }
      cudaFree(c->tile_cnt[k]); cudaFree(c->tile_pre[k]);
      c->tile_cnt[k] = nullptr; c->tile_pre[k] = nullptr; c->tile_cap[k] = 0;
      CK(cudaMalloc(&c->tile_cnt[k], sizeof(unsigned int) * want_t[k]));
      CK(cudaMalloc(&c->tile_pre[k], sizeof(unsigned int) * want_t[k]));
      CK(cudaMemsetAsync(c->tile_cnt[k], 0, sizeof(unsigned int) * want_t[k], s));
      c->tile_cap[k] = want_t[k];
    }
    if (want_r[k] > c->rec_cap[k]) {
      if (!sync_done) { CK(cudaStreamSynchronize(s)); sync_done = true; }
      cudaFree(c->rec[k]);
      c->rec[k] = nullptr; c->rec_cap[k] = 0;
      CK(cudaMalloc(&c->rec[k], rbytes[k] * want_r[k]));
      CK(cudaMemsetAsync(c->rec[k], 0, rbytes[k] * want_r[k], s));
      if (k == 0) {
        cudaFree(c->holes);
        c->holes = nullptr;
        CK(cudaMalloc(&c->holes, sizeof(unsigned int) * want_r[0]));
      }
      c->rec_cap[k] = want_r[k];
    }
  }
  if (sync_done) CK(cudaStreamSynchronize(s));
  return QED_OK;
}

extern "C" qed_status particles_create(qed_ctx* c, qed_species sp, const qed_soa* b, uint64_t n, uint64_t cap,
                                       qed_precision prec, void* stream, qed_particles** out) {
  if (!out) FAIL(QED_ERR_INVALID_ARG, "particles_create: out is NULL");
  *out = nullptr;
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "particles_create: invalid context");
  if (!b) FAIL(QED_ERR_INVALID_ARG, "particles_create: buffers is NULL");
  if (sp < QED_ELECTRON || sp > QED_PHOTON) FAIL(QED_ERR_INVALID_ARG, "particles_create: bad species %d", (int)sp);
  if (prec != QED_PREC_F64 && prec != QED_PREC_MIXED) FAIL(QED_ERR_INVALID_ARG, "particles_create: bad precision");
  if (n > cap) FAIL(QED_ERR_INVALID_ARG, "particles_create: n (%llu) > capacity (%llu)",
                    (unsigned long long)n, (unsigned long long)cap);
  if (cap > (1ull << 32) - 256)
    FAIL(QED_ERR_INVALID_ARG, "particles_create: capacity must not exceed 2^32 - 256");
  if (cap > 0) {
    const void* req[] = {b->x, b->y, b->z, b->px, b->py, b->pz, b->s1, b->s2, b->s3, b->w, b->id};
    for (const void* p : req)
      if (!p) FAIL(QED_ERR_INVALID_ARG, "particles_create: a required array is NULL");
    if (sp == QED_PHOTON && !b->theta) FAIL(QED_ERR_INVALID_ARG, "particles_create: photons need theta");
  }
  cudaStream_t s = S(stream);
  if (cap > c->cap_seen[sp]) c->cap_seen[sp] = cap;
  qed_status r = grow_scratch(c, s);
  if (r != QED_OK) return r;
  qed_particles* p = (qed_particles*)calloc(1, sizeof(qed_particles));
  p->ctx = c;
  p->species = sp;
  p->prec = prec;
  p->soa = *b;
  p->cap = cap;
  unsigned long long nn = n;
  CK(cudaMemcpyAsync(&c->st->n_live[sp], &nn, sizeof(nn), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  *out = p;
  return QED_OK;
}

extern "C" qed_status particles_count(const qed_particles* p, uint64_t* n, void* stream) {
  if (!p || !n) FAIL(QED_ERR_INVALID_ARG, "particles_count: NULL argument");
  if (!p->ctx || !p->ctx->alive) FAIL(QED_ERR_NOT_INITIALIZED, "particles_count: context destroyed");
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, &p->ctx->st->n_live[p->species], sizeof(v), cudaMemcpyDeviceToHost, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  *n = v;
  return QED_OK;
}

extern "C" qed_status particles_set_count(qed_particles* p, uint64_t n, void* stream) {
  if (!p) FAIL(QED_ERR_INVALID_ARG, "particles_set_count: NULL");
  if (n > p->cap) FAIL(QED_ERR_INVALID_ARG, "particles_set_count: n > capacity");
  static thread_local unsigned long long hv;
  hv = n;
  CK(cudaMemcpyAsync(&p->ctx->st->n_live[p->species], &hv, sizeof(hv), cudaMemcpyHostToDevice, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  return QED_OK;
}

extern "C" qed_status particles_destroy(qed_particles* p) {
  if (!p) FAIL(QED_ERR_INVALID_ARG, "particles_destroy: NULL");
  free(p);
  return QED_OK;
}

extern "C" qed_status qed_set_next_id(qed_ctx* c, uint64_t id, void* stream) {
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_set_next_id: invalid context");
  static thread_local unsigned long long hv;
  hv = id;
  CK(cudaMemcpyAsync(&c->st->next_id, &hv, sizeof(hv), cudaMemcpyHostToDevice, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  return QED_OK;
}

extern "C" qed_status qed_get_next_id(qed_ctx* c, uint64_t* id, void* stream) {
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_get_next_id: invalid context");
  if (!id) FAIL(QED_ERR_INVALID_ARG, "qed_get_next_id: NULL");
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, &c->st->next_id, sizeof(v), cudaMemcpyDeviceToHost, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  *id = v;
  return QED_OK;
}

extern "C" qed_status qed_read_status(qed_ctx* c, uint32_t* status, int clear, void* stream) {
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_read_status: invalid context");
  if (!status) FAIL(QED_ERR_INVALID_ARG, "qed_read_status: NULL");
  unsigned int v = 0;
  CK(cudaMemcpyAsync(&v, &c->st->status, sizeof(v), cudaMemcpyDeviceToHost, S(stream)));
  if (clear) CK(cudaMemsetAsync(&c->st->status, 0, sizeof(unsigned int), S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  *status = v;
  return QED_OK;
}

static void fill_species(SpeciesArgs& a, const qed_particles* p) {
  memset(&a, 0, sizeof(a));
  if (!p) return;
  a.x = (double*)p->soa.x; a.y = (double*)p->soa.y; a.z = (double*)p->soa.z;
  a.px = p->soa.px; a.py = p->soa.py; a.pz = p->soa.pz;
  a.s1 = p->soa.s1; a.s2 = p->soa.s2; a.s3 = p->soa.s3;
  a.theta = p->soa.theta; a.w = p->soa.w; a.id = p->soa.id;
  a.cap = p->cap;
  a.present = p->cap > 0 ? 1 : 0;
}

namespace qedk {
// float(t - phi0) and float(t mod 2 pi), formed in FP64 with one explicit fma so that the
// batched kernels' clock advance on the device gives the same values
void step_time_floats(double t, double phi0, float* t_rel, float* t_mod) {
  *t_rel = (float)(t - phi0);
  *t_mod = (float)std::fma(-kTwoPi, std::floor(t / kTwoPi), t);
}

void philox_key_schedule(uint64_t seed, unsigned int rk[20]) {
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = (uint32_t)seed + (uint32_t)r * kPhiloxW0;
    rk[2 * r + 1] = (uint32_t)(seed >> 32) + (uint32_t)r * kPhiloxW1;
  }
}

void set_medium_args(StepArgs& a, const qed_ctx* c) {
  if (!c->has_medium) return;
  const double* C = static_cast<const double*>(c->med_buf);
  a.med_c = C;
  a.med_tot = reinterpret_cast<const float*>(C + 2 * (size_t)kNmg * kNms);
  a.med_nar2 = c->med.n * kAlpha * kR0n * kR0n;
  a.med_lo = c->med.lo;
  a.med_hi = c->med.hi;
  a.med_kmin = c->med.k_min;
  a.med_axis = c->med.axis;
}

void fill_ensemble(EnsArgs& E, const qed_particles* e, const qed_particles* pos, const qed_particles* ph,
                   const qed_fields* f, double t, uint64_t seed, uint32_t step, DevState* st,
                   qed_step_stats* stats) {
  memset(&E, 0, sizeof(E));
  fill_species(E.sp[0], e);
  fill_species(E.sp[1], pos);
  fill_species(E.sp[2], ph);
  E.f = *f;
  E.t = t;
  E.seed = seed;
  philox_key_schedule(seed, E.rk);
  E.step = step;
  E.st = st;
  E.user_stats = stats;
  const double len = f->len > 0.0 ? f->len : 1.0;
  E.inv_len = 1.0 / len;
  E.ff.inv_len = (float)E.inv_len;
  step_time_floats(t, f->phi0, &E.ff.t_rel, &E.ff.t_mod);
  E.ff.a0 = (float)f->a0;
  E.ff.w0 = (float)f->w0;
  E.ff.zf = (float)f->zf;
  E.ff.zr = (float)(0.5 * f->w0 * f->w0);
  E.ff.inv_zr = f->w0 > 0.0 ? (float)(2.0 / (f->w0 * f->w0)) : 0.0f;
  E.ff.inv_w02 = f->w0 > 0.0 ? (float)(1.0 / (f->w0 * f->w0)) : 0.0f;
  if (f->kind == QED_FIELD_GRID2D && f->dx > 0.0 && f->dy > 0.0) {
    // float splits hi + lo of the grid constants: the mixed path forms cell coordinates as
    // an integer node plus a float offset from them (no FP64 arithmetic on the device)
    auto split = [](double v, float& h, float& l) {
      h = (float)v;
      l = (float)(v - (double)h);
    };
    split(1.0 / f->dx, E.ff.gix, E.ff.gix_lo);
    split(1.0 / f->dy, E.ff.giy, E.ff.giy_lo);
    const double ox = f->x0 / f->dx, oy = f->y0 / f->dy;
    const double gx = std::floor(ox), gy = std::floor(oy);
    E.ff.gox_i = (int)gx;
    E.ff.goy_i = (int)gy;
    split(ox - gx, E.ff.gox, E.ff.gox_lo);
    split(oy - gy, E.ff.goy, E.ff.goy_lo);
  }
}
}  // namespace qedk

namespace qedk {
qed_status check_flag_bits(uint32_t flags, const char* who) {
  if (flags & ~kAllFlags) FAIL(QED_ERR_INVALID_ARG, "%s: unknown flag bits 0x%x", who, flags & ~kAllFlags);
  if ((flags & (QED_F_LL | QED_F_MLL | QED_F_MBMT)) && (flags & QED_F_NCS))
    FAIL(QED_ERR_INVALID_ARG, "%s: the radiative pusher (LL, MLL, MBMT) and the NCS Monte Carlo count the same "
         "radiation: choose one", who);
  if ((flags & QED_F_LL) && (flags & QED_F_MLL)) FAIL(QED_ERR_INVALID_ARG, "%s: QED_F_LL and QED_F_MLL exclude each other", who);
  if ((flags & (QED_F_BREMS | QED_F_BH)) && (flags & (QED_F_LL | QED_F_MLL | QED_F_MBMT)))
    FAIL(QED_ERR_INVALID_ARG, "%s: the matter processes run with the Monte Carlo step, not with the radiative pusher", who);
  return QED_OK;
}

qed_status check_mlp_flag(const qed_ctx* c, uint32_t flags, qed_precision prec, const char* who) {
  if (!(flags & QED_F_MLP)) return QED_OK;
  if (prec != QED_PREC_MIXED) FAIL(QED_ERR_INVALID_ARG, "%s: the learned sampler runs on the mixed path only", who);
  const qed_ctx* o = c->owner ? c->owner : c;
  if (!o->mlp_ready) FAIL(QED_ERR_NOT_INITIALIZED, "%s: the learned sampler has no parameters (qed_mlp_train)", who);
  return QED_OK;
}

qed_status check_deposit(uint32_t flags, const qed_fields* f, const char* who) {
  if (!(flags & QED_F_DEPOSIT)) return QED_OK;
  if (f->kind != QED_FIELD_GRID2D || !f->gJx || !f->gJy || !f->gJz)
    FAIL(QED_ERR_INVALID_ARG, "%s: QED_F_DEPOSIT needs a grid field with current arrays", who);
  return QED_OK;
}

qed_status check_fields(const qed_fields* f, const char* who) {
  // every parameter the kind uses must be finite: a NaN or inf here would reach every
  // particle of the step
  bool finite = true;
  if (f->kind == QED_FIELD_UNIFORM)
    for (int k = 0; k < 3; ++k) finite = finite && std::isfinite(f->E[k]) && std::isfinite(f->B[k]);
  if (f->kind == QED_FIELD_PLANE || f->kind == QED_FIELD_GAUSS)
    finite = std::isfinite(f->a0) && std::isfinite(f->phi0) && std::isfinite(f->len) &&
             (f->kind == QED_FIELD_PLANE || (std::isfinite(f->w0) && std::isfinite(f->zf)));
  if (f->kind == QED_FIELD_GRID2D)
    finite = std::isfinite(f->dx) && std::isfinite(f->dy) && std::isfinite(f->x0) && std::isfinite(f->y0);
  if (!finite) FAIL(QED_ERR_INVALID_ARG, "%s: non-finite field parameter", who);
  switch (f->kind) {
    case QED_FIELD_NONE:
    case QED_FIELD_UNIFORM:
      break;
    case QED_FIELD_PLANE:
      if (!(f->len > 0.0)) FAIL(QED_ERR_INVALID_ARG, "%s: envelope length must be positive", who);
      break;
    case QED_FIELD_GAUSS:
      if (!(f->len > 0.0) || !(f->w0 > 0.0)) FAIL(QED_ERR_INVALID_ARG, "%s: len and w0 must be positive", who);
      break;
    case QED_FIELD_GRID2D:
      if (!f->gEx || !f->gEy || !f->gEz || !f->gBx || !f->gBy || !f->gBz)
        FAIL(QED_ERR_INVALID_ARG, "%s: grid arrays must be non-NULL", who);
      if (f->periodic != 0 && f->periodic != 1) FAIL(QED_ERR_INVALID_ARG, "%s: periodic must be 0 or 1", who);
      if (f->nx < 1 || f->ny < 1 || !(f->dx > 0) || !(f->dy > 0)) FAIL(QED_ERR_INVALID_ARG, "%s: bad grid geometry", who);
      break;
    default:
      FAIL(QED_ERR_INVALID_ARG, "%s: unknown field kind %d", who, f->kind);
  }
  return QED_OK;
}
}  // namespace qedk

static qed_status validate_step(qed_ctx* c, qed_particles* e, qed_particles* pos, qed_particles* ph,
                                const qed_fields* f, double dt, uint32_t flags, qed_precision* prec) {
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_step: invalid context");
  if (c->pending) FAIL(QED_ERR_INVALID_ARG, "qed_step: a sharded step is between qed_step_begin and qed_step_end");
  if (!f) FAIL(QED_ERR_INVALID_ARG, "qed_step: fields is NULL");
  if (!(dt > 0.0) || !std::isfinite(dt)) FAIL(QED_ERR_INVALID_ARG, "qed_step: dt must be positive and finite");
  {
    const qed_status rf = check_flag_bits(flags, "qed_step");
    if (rf != QED_OK) return rf;
  }
  const qed_particles* all[3] = {e, pos, ph};
  const qed_species want[3] = {QED_ELECTRON, QED_POSITRON, QED_PHOTON};
  int have = -1;
  for (int k = 0; k < 3; ++k) {
    if (!all[k]) continue;
    if (all[k]->ctx != c) FAIL(QED_ERR_INVALID_ARG, "qed_step: particle set from another context");
    if (all[k]->species != want[k]) FAIL(QED_ERR_INVALID_ARG, "qed_step: argument %d has the wrong species", k);
    if (have >= 0 && (int)all[k]->prec != have) FAIL(QED_ERR_INVALID_ARG, "qed_step: mixed precisions");
    have = (int)all[k]->prec;
  }
  *prec = have < 0 ? QED_PREC_F64 : (qed_precision)have;
  if ((flags & QED_F_NBW) && (!e || !pos)) FAIL(QED_ERR_INVALID_ARG, "qed_step: NBW needs e- and e+ sets");
  qed_status r_ = check_mlp_flag(c, flags, *prec, "qed_step");
  if (r_ != QED_OK) return r_;
  r_ = check_fields(f, "qed_step");
  if (r_ != QED_OK) return r_;
  r_ = check_deposit(flags, f, "qed_step");
  if (r_ != QED_OK) return r_;
  if ((flags & (QED_F_BREMS | QED_F_BH)) && !c->has_medium)
    FAIL(QED_ERR_INVALID_ARG, "qed_step: QED_F_BREMS / QED_F_BH need a medium (qed_set_medium)");
  if ((flags & QED_F_BH) && (!e || !pos)) FAIL(QED_ERR_INVALID_ARG, "qed_step: Bethe-Heitler pairs need e- and e+ sets");
  const unsigned long long tp = ph ? tiles_of(ph->cap) : 0;
  const unsigned long long tl = (e ? tiles_of(e->cap) : 0) + (pos ? tiles_of(pos->cap) : 0);
  if (tp > c->tile_cap[0] || tl > c->tile_cap[1] || !c->rec[0] || !c->rec[1])
    FAIL(QED_ERR_INVALID_ARG, "qed_step: particle sets larger than the context's scratch");
  return QED_OK;
}

// the launch arguments of one step on the context's scratch
static void step_args(StepArgs& a, qed_ctx* c, qed_particles* e, qed_particles* pos, qed_particles* ph,
                      const qed_fields* f, double t, double dt, uint64_t seed, uint32_t step, uint32_t flags,
                      qed_step_stats* dev_stats, qed_precision prec) {
  memset(&a, 0, sizeof(a));
  fill_ensemble(a.e0, e, pos, ph, f, t, seed, step, c->st, dev_stats);
  a.dt = dt;
  a.fdt = (float)dt;
  a.flags = flags;
  a.tables = prec == QED_PREC_F64 ? (const void*)c->tab64 : (const void*)c->tab32;
  a.mlp = (c->owner ? c->owner : c)->mlp;
  a.st = c->st;
  for (int k = 0; k < 2; ++k) {
    a.tile_cnt[k] = c->tile_cnt[k];
    a.tile_pre[k] = c->tile_pre[k];
    a.rec[k] = c->rec[k];
    a.rec_cap[k] = c->rec_cap[k];
  }
  a.holes = c->holes;
  set_medium_args(a, c);
}

extern "C" qed_status qed_step_begin(qed_ctx* c, qed_particles* e, qed_particles* pos, qed_particles* ph,
                                     const qed_fields* f, double t, double dt, uint64_t seed, uint32_t step,
                                     uint32_t flags, qed_step_stats* dev_stats, uint64_t* dev_counts, void* stream) {
  const qedk::NvtxRange nvtx_range("qed_step_begin");
  qed_precision prec;
  qed_status r = validate_step(c, e, pos, ph, f, dt, flags, &prec);
  if (r != QED_OK) return r;
  if (!dev_counts) FAIL(QED_ERR_INVALID_ARG, "qed_step_begin: dev_counts is NULL");
  if (c->timing) FAIL(QED_ERR_INVALID_ARG, "qed_step_begin: per-kernel timing is on");
  StepArgs& a = c->pend;
  step_args(a, c, e, pos, ph, f, t, dt, seed, step, flags, dev_stats, prec);
  a.shard_counts = reinterpret_cast<unsigned long long*>(dev_counts);
  const int pi = prec == QED_PREC_F64 ? 0 : 1;
  StreamSet ss{c->side, c->fork, c->join, nullptr};
  r = launch_step(a, prec, c->nblk[pi], S(stream), ss, kStepBegin);
  if (r != QED_OK) return r;
  c->pend_prec = prec;
  c->pending = 1;
  return QED_OK;
}

extern "C" qed_status qed_step_end(qed_ctx* c, const uint64_t* dev_all, int rank, int world, void* stream) {
  const qedk::NvtxRange nvtx_range("qed_step_end");
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_step_end: invalid context");
  if (!c->pending) FAIL(QED_ERR_INVALID_ARG, "qed_step_end: no step begun (qed_step_begin)");
  if (!dev_all) FAIL(QED_ERR_INVALID_ARG, "qed_step_end: dev_all is NULL");
  if (world < 1 || rank < 0 || rank >= world)
    FAIL(QED_ERR_INVALID_ARG, "qed_step_end: rank %d outside [0, %d)", rank, world);
  StepArgs& a = c->pend;
  a.shard_all = reinterpret_cast<const unsigned long long*>(dev_all);
  a.shard_rank = rank;
  a.shard_world = world;
  const int pi = c->pend_prec == QED_PREC_F64 ? 0 : 1;
  StreamSet ss{c->side, c->fork, c->join, nullptr};
  c->pending = 0;
  return launch_step(a, c->pend_prec, c->nblk[pi], S(stream), ss, kStepEnd);
}

extern "C" qed_status qed_step(qed_ctx* c, qed_particles* e, qed_particles* pos, qed_particles* ph,
                               const qed_fields* f, double t, double dt, uint64_t seed, uint32_t step,
                               uint32_t flags, qed_step_stats* dev_stats, void* stream) {
  const qedk::NvtxRange nvtx_range("qed_step");
  qed_precision prec;
  qed_status r = validate_step(c, e, pos, ph, f, dt, flags, &prec);
  if (r != QED_OK) return r;
  StepArgs a;
  step_args(a, c, e, pos, ph, f, t, dt, seed, step, flags, dev_stats, prec);
  const int pi = prec == QED_PREC_F64 ? 0 : 1;
  // per-kernel timing runs the passes one after the other, so that each duration is the
  // kernel's own (no overlap of the lepton pass with the photon chain)
  StreamSet ss{c->timing ? nullptr : c->side, c->fork, c->join, c->timing ? c->tev : nullptr};
  r = launch_step(a, prec, c->nblk[pi], S(stream), ss);
  if (r != QED_OK || !c->timing) return r;
  CK(cudaEventSynchronize(c->tev[3]));
  CK(cudaEventSynchronize(c->tev[5]));
  float m[3] = {0, 0, 0}, tot = 0;
  CK(cudaEventElapsedTime(&m[0], c->tev[0], c->tev[1]));
  CK(cudaEventElapsedTime(&m[1], c->tev[4], c->tev[5]));
  CK(cudaEventElapsedTime(&tot, c->tev[1], c->tev[3]));   // event kernels and the lepton pass
  c->tms[0] += m[0];
  c->tms[1] += m[1];
  c->tms[2] += tot - m[1];
  c->tsteps += 1;
  return QED_OK;
}

extern "C" qed_status qed_set_timing(qed_ctx* c, int enable) {
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_set_timing: invalid context");
  if (enable && !c->tev[0]) {
    for (int k = 0; k < 6; ++k) CK(cudaEventCreate(&c->tev[k]));
  }
  c->timing = enable ? 1 : 0;
  return QED_OK;
}

extern "C" qed_status qed_get_timing(qed_ctx* c, double ms[3], uint64_t* steps) {
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_get_timing: invalid context");
  if (!ms || !steps) FAIL(QED_ERR_INVALID_ARG, "qed_get_timing: NULL output");
  for (int k = 0; k < 3; ++k) ms[k] = c->tms[k];
  *steps = c->tsteps;
  c->tms[0] = c->tms[1] = c->tms[2] = 0.0;
  c->tsteps = 0;
  return QED_OK;
}

static size_t elem(qed_precision p) { return p == QED_PREC_F64 ? 8 : 4; }

static qed_status copy_soa(const qed_soa* dst, const qed_soa* src, unsigned long long n, qed_precision prec,
                           bool photon, cudaMemcpyKind kind, cudaStream_t s) {
  if (n == 0) return QED_OK;
  const size_t r = elem(prec);
  void* const d8[3] = {dst->x, dst->y, dst->z};
  void* const s8[3] = {src->x, src->y, src->z};
  for (int k = 0; k < 3; ++k) CK(cudaMemcpyAsync(d8[k], s8[k], 8 * n, kind, s));
  void* const dr[7] = {dst->px, dst->py, dst->pz, dst->s1, dst->s2, dst->s3, dst->w};
  void* const sr[7] = {src->px, src->py, src->pz, src->s1, src->s2, src->s3, src->w};
  for (int k = 0; k < 7; ++k) CK(cudaMemcpyAsync(dr[k], sr[k], r * n, kind, s));
  if (photon) CK(cudaMemcpyAsync(dst->theta, src->theta, r * n, kind, s));
  CK(cudaMemcpyAsync(dst->id, src->id, 8 * n, kind, s));
  return QED_OK;
}

extern "C" qed_status qed_step_host(qed_ctx* c, qed_particles* e, qed_particles* pos, qed_particles* ph,
                                    const qed_soa* he, const qed_soa* hp, const qed_soa* hg, uint64_t n_host[3],
                                    const qed_fields* f, double t, double dt, uint64_t seed, uint32_t step,
                                    uint32_t flags, void* stream) {
  const qedk::NvtxRange nvtx_range("qed_step_host");
  qed_precision prec;
  qed_status r = validate_step(c, e, pos, ph, f, dt, flags, &prec);
  if (r != QED_OK) return r;
  if (!n_host) FAIL(QED_ERR_INVALID_ARG, "qed_step_host: n_host is NULL");
  qed_particles* dev[3] = {e, pos, ph};
  const qed_soa* host[3] = {he, hp, hg};
  cudaStream_t s = S(stream);
  for (int k = 0; k < 3; ++k) {
    if (!dev[k]) continue;
    if (!host[k]) FAIL(QED_ERR_INVALID_ARG, "qed_step_host: host set %d missing", k);
    if (n_host[k] > dev[k]->cap) FAIL(QED_ERR_INVALID_ARG, "qed_step_host: n_host[%d] > capacity", k);
  }
  static thread_local unsigned long long counts[3];
  for (int k = 0; k < 3; ++k) {
    if (!dev[k]) continue;
    r = copy_soa(&dev[k]->soa, host[k], n_host[k], prec, k == 2, cudaMemcpyHostToDevice, s);
    if (r != QED_OK) return r;
    counts[k] = n_host[k];
    CK(cudaMemcpyAsync(&c->st->n_live[k], &counts[k], sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
  }
  r = qed_step(c, e, pos, ph, f, t, dt, seed, step, flags, nullptr, stream);
  if (r != QED_OK) return r;
  CK(cudaMemcpyAsync(counts, c->st->n_live, sizeof(counts), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < 3; ++k) {
    if (!dev[k]) continue;
    r = copy_soa(host[k], &dev[k]->soa, counts[k], prec, k == 2, cudaMemcpyDeviceToHost, s);
    if (r != QED_OK) return r;
    n_host[k] = counts[k];
  }
  CK(cudaStreamSynchronize(s));
  return QED_OK;
}

extern "C" qed_status qed_philox_blocks(const uint32_t* ctr, uint64_t key, uint32_t* out, uint64_t n, void* stream) {
  if (n == 0) return QED_OK;
  if (!ctr || !out) FAIL(QED_ERR_INVALID_ARG, "qed_philox_blocks: NULL buffer");
  if (n > (1ull << 40)) FAIL(QED_ERR_INVALID_ARG, "qed_philox_blocks: n too large");
  CK(launch_philox_blocks(ctr, key, out, n, S(stream)));
  return QED_OK;
}

extern "C" qed_status qed_copy_table(qed_ctx* c, int which, double* host, uint64_t cap, uint64_t* len, void* stream) {
  if (!c || !c->alive) FAIL(QED_ERR_NOT_INITIALIZED, "qed_copy_table: invalid context");
  if (!len) FAIL(QED_ERR_INVALID_ARG, "qed_copy_table: len is NULL");
  size_t off, n;
  switch (which) {
    case 0: off = kOffKV; n = 6 * (size_t)kNK; break;
    case 1: off = kOffRA; n = 2 * (size_t)kNR; break;
    case 2: off = kOffCY; n = 4 * (size_t)kNCX * kNCT; break;
    case 3: off = kOffT0; n = 2 * (size_t)kNBX; break;
    case 4: off = kOffBY; n = 4 * (size_t)kNBX * kNBT; break;
    case 5: off = kOffMP; n = 2 * (size_t)kNV; break;
    case 6: off = kOffRR; n = 4 * (size_t)kNR; break;
    case 7: off = kOffCoefVB; n = kTab32Len - kOffCoefVB; break;
    default: FAIL(QED_ERR_INVALID_ARG, "qed_copy_table: which must be 0..7");
  }
  *len = n;
  if (!host) return QED_OK;
  if (cap < n) FAIL(QED_ERR_INVALID_ARG, "qed_copy_table: cap %llu < %llu", (unsigned long long)cap,
                    (unsigned long long)n);
  if (which == 7) {   // float block of the mixed path
    std::vector<float> tmp(n);
    CK(cudaMemcpyAsync(tmp.data(), c->tab32 + off, n * sizeof(float), cudaMemcpyDeviceToHost, S(stream)));
    CK(cudaStreamSynchronize(S(stream)));
    for (size_t i = 0; i < n; ++i) host[i] = (double)tmp[i];
    return QED_OK;
  }
  CK(cudaMemcpyAsync(host, c->tab64 + off, n * sizeof(double), cudaMemcpyDeviceToHost, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  return QED_OK;
}
