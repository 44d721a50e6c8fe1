// qed_step.cu -- one step of one ensemble: launch sequence of the kernels of
// qed_kernels.cuh (single-ensemble instantiations) and the persistent grid sizes.
#include "qed_kernels.cuh"

namespace qedk {

size_t nbw_rec_bytes(qed_precision p) { return p == QED_PREC_F64 ? sizeof(NbwRec<double>) : sizeof(NbwRec<float>); }
size_t ncs_rec_bytes(qed_precision p) { return p == QED_PREC_F64 ? sizeof(NcsRec<double>) : sizeof(NcsRec<float>); }

// Photon pass on the caller's stream; the lepton pass on the context's side stream (forked
// after all earlier work on the caller's stream, joined before the scans): the two passes
// touch disjoint particles, and everything that needs both (births, refills, pair events)
// is in k_events.
template <typename R>
static void launch_lepton(const StepArgs& a, int grid, cudaStream_t s) {
  const bool rad = a.flags & (QED_F_LL | QED_F_MLL | QED_F_MBMT), dep = a.flags & QED_F_DEPOSIT;
  const bool med = a.flags & QED_F_BREMS;
  if (med && dep) k_lepton<R, false, true, false, true, true><<<grid, kTile, 0, s>>>(a);
  else if (med) k_lepton<R, false, true, false, false, true><<<grid, kTile, 0, s>>>(a);
  else if (rad && dep) k_lepton<R, false, true, true, true><<<grid, kTile, 0, s>>>(a);
  else if (rad) k_lepton<R, false, true, true><<<grid, kTile, 0, s>>>(a);
  else if (dep) k_lepton<R, false, true, false, true><<<grid, kTile, 0, s>>>(a);
  else k_lepton<R, false, true><<<grid, kTile, 0, s>>>(a);
}

static qed_status launch_status() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("step launch failed: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  return QED_OK;
}

// the event kernel, which closes the step
template <typename R>
static qed_status launch_events(const StepArgs& a, const int* nb, cudaStream_t s, bool pdl, const StreamSet& ss) {
  if constexpr (sizeof(R) == 4) {
    if (a.flags & QED_F_MLP) launch_k(k_events_mlp<false>, nb[2] * 2, kMlpRows, s, pdl, a);
    else launch_k(k_events<R, false>, nb[2], kTile, s, pdl, a);
  } else {
    launch_k(k_events<R, false>, nb[2], kTile, s, pdl, a);
  }
  if (ss.tev) cudaEventRecord(ss.tev[3], s);
  return launch_status();
}

template <typename R>
static qed_status launch_t(const StepArgs& a, const int* nb, cudaStream_t s, const StreamSet& ss, StepPart part) {
  const bool fork = ss.side != nullptr;
  const bool pdl = ss.tev == nullptr;   // timing events between kernels would break the pairs
  if (part == kStepEnd) {
    k_shard_ids<<<1, 32, 0, s>>>(a);
    return launch_events<R>(a, nb, s, pdl, ss);
  }
  if (ss.tev) cudaEventRecord(ss.tev[0], s);
  if (fork) {
    cudaEventRecord(ss.fork, s);
    cudaStreamWaitEvent(ss.side, ss.fork, 0);
    if (ss.tev) cudaEventRecord(ss.tev[4], ss.side);
    launch_lepton<R>(a, nb[1], ss.side);
    if (ss.tev) cudaEventRecord(ss.tev[5], ss.side);
    cudaEventRecord(ss.join, ss.side);
  }
  if (a.flags & QED_F_BH) k_photon<R, false, true, true><<<nb[0], kTile, 0, s>>>(a);
  else k_photon<R, false, true><<<nb[0], kTile, 0, s>>>(a);
  if (ss.tev) cudaEventRecord(ss.tev[1], s);
  if (fork) {
    cudaStreamWaitEvent(s, ss.join, 0);
  } else {
    if (ss.tev) cudaEventRecord(ss.tev[4], s);
    launch_lepton<R>(a, nb[1], s);
    if (ss.tev) cudaEventRecord(ss.tev[5], s);
  }
  k_scan<R, false><<<2, kScanThreads, 0, s>>>(a, -1);   // both scans, after both passes
  if (part == kStepBegin) {
    k_shard_counts<<<1, 32, 0, s>>>(a);
    return launch_status();
  }
  return launch_events<R>(a, nb, s, pdl, ss);
}

qed_status launch_step(const StepArgs& a, qed_precision prec, const int* nblk, cudaStream_t s, const StreamSet& ss,
                       StepPart part) {
  return prec == QED_PREC_F64 ? launch_t<double>(a, nblk, s, ss, part) : launch_t<float>(a, nblk, s, ss, part);
}

qed_status step_grid_sizes(qed_precision prec, int* nblk) {
  int dev = 0, sms = 0, b0 = 0, b1 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (prec == QED_PREC_F64) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_photon<double, false, true>, kTile, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_lepton<double, false, true>, kTile, 0);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_photon<float, false, true>, kTile, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_lepton<float, false, true>, kTile, 0);
  }
  if (e != cudaSuccess || b0 < 1 || b1 < 1) {
    set_error("occupancy query failed: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  nblk[0] = sms * b0;
  nblk[1] = sms * b1;
  nblk[2] = sms * 2;   // event kernels: grid-stride over the logged events
  return QED_OK;
}

}  // namespace qedk
