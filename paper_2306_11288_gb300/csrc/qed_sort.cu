// qed_sort.cu -- cell sort of a particle set on a 2D grid (qed_sort_cells).
//
// A PIC code keeps its particles ordered by cell so that a warp's field gathers and current
// deposits touch a few cache lines instead of 32 (on the 3e7-electron grid workload the
// step runs 1.6x faster with cell-ordered electrons).  The order is by 32x32-cell tile, and
// inside a tile by cell, row-major; particles outside a bounded grid go last.  The sort is
// stable (equal cells keep their order), so it is deterministic and reproducible.
//
// Least-significant-digit radix sort of (key, index) pairs with 8-bit digits over the key
// bits in use, then a gather of every array of the set through the sorted indices.  Each
// pass: a digit histogram per block over a contiguous chunk of the input (k_sort_hist), an
// exclusive scan of the (digit, block) counts in digit-major order (k_sort_scan), and a
// stable scatter in which every block walks its chunk in order and ranks equal digits
// inside a warp with __match_any_sync (k_sort_scatter).  The live count is read on the
// device: no host synchronisation.
#include <cmath>

#include "qed_common.cuh"
#include "qed_internal.h"

namespace qedk {

constexpr int kSortThreads = 256;
constexpr int kSortBlocks = 512;
constexpr int kSortItems = 8;    // sub-tiles of 256 keys per scatter iteration
constexpr int kGroup = 4;        // arrays gathered by one launch

__device__ __forceinline__ unsigned long long sort_chunk(unsigned long long n) {
  const unsigned long long c = (n + kSortBlocks - 1) / kSortBlocks;
  return (c + kSortThreads - 1) / kSortThreads * kSortThreads;
}

// cell of a coordinate: floor((x - x0) * (1/dx)), both operations rounded in double, the
// floor taken by the conversion itself (three FP64 operations, no division)
__device__ __forceinline__ long long cell_index(double x, double x0, double inv) {
  return __double2ll_rd((x - x0) * inv);
}

__global__ void __launch_bounds__(kSortThreads) k_sort_keys(const unsigned long long* n_live, qed_fields f,
                                                            double inv_dx, double inv_dy, const double* x,
                                                            const double* y, unsigned int* key, unsigned int* idx,
                                                            unsigned int key_out) {
  const unsigned long long n = *n_live;
  const int tx = (f.nx + 31) >> 5;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    long long ci = cell_index(x[i], f.x0, inv_dx), cj = cell_index(y[i], f.y0, inv_dy);
    unsigned int k = key_out;
    if (f.periodic) {
      // wrap: one period either way without a division, the general case with one
      if (ci < 0 && ci >= -(long long)f.nx) ci += f.nx;
      else if (ci >= f.nx && ci < 2ll * f.nx) ci -= f.nx;
      else if (ci < 0 || ci >= f.nx) { ci %= f.nx; ci += ci < 0 ? f.nx : 0; }
      if (cj < 0 && cj >= -(long long)f.ny) cj += f.ny;
      else if (cj >= f.ny && cj < 2ll * f.ny) cj -= f.ny;
      else if (cj < 0 || cj >= f.ny) { cj %= f.ny; cj += cj < 0 ? f.ny : 0; }
    }
    // a NaN position converts to the most negative integer: outside
    if (ci >= 0 && ci < f.nx && cj >= 0 && cj < f.ny)
      k = (unsigned int)((((cj >> 5) * tx + (ci >> 5)) << 10) + ((cj & 31) << 5) + (ci & 31));
    key[i] = k;
    idx[i] = (unsigned int)i;
  }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const unsigned long long* n_live, const unsigned int* key,
                                                            int shift, unsigned int* counts) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const unsigned long long n = *n_live, c = sort_chunk(n);
  const unsigned long long b0 = blockIdx.x * c, b1 = b0 + c < n ? b0 + c : n;
  for (unsigned long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
  __syncthreads();
  counts[threadIdx.x * kSortBlocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of the 256 * kSortBlocks counts in place, one block of 1024 threads, in
// chunks of 8192: each thread takes 8 consecutive counts (two 16-byte loads, so a warp
// reads 1 KB in one piece), a block scan of the thread sums, the running total carried
__global__ void __launch_bounds__(1024) k_sort_scan(unsigned int* counts) {
  constexpr int kN = 256 * kSortBlocks, kPer = 8, kChunk = 1024 * kPer;
  static_assert(kN % kChunk == 0, "whole chunks");
  __shared__ unsigned int s_w[32];
  __shared__ unsigned int s_run;
  const unsigned int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  for (int base = 0; base < kN; base += kChunk) {
    uint4* p = reinterpret_cast<uint4*>(counts + base + threadIdx.x * kPer);
    const uint4 a = p[0], b = p[1];
    unsigned int v[kPer] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    unsigned int t = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) t += v[j];
    unsigned int incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned int w = s_w[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= (unsigned)o) w += u;
      }
      s_w[lane] = w;
    }
    __syncthreads();
    unsigned int run = s_run + (warp ? s_w[warp - 1] : 0u) + incl - t;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const unsigned int e = run;
      run += v[j];
      v[j] = e;
    }
    p[0] = make_uint4(v[0], v[1], v[2], v[3]);
    p[1] = make_uint4(v[4], v[5], v[6], v[7]);
    __syncthreads();
    if (threadIdx.x == 0) s_run += s_w[31];
    __syncthreads();
  }
}

// Stable scatter of one digit.  Every block walks its chunk in order, kIter keys per
// iteration (the next iteration's keys in flight meanwhile); warp w owns the iteration's
// keys w*256 .. w*256+255, kSortItems per lane (item j of lane l is key w*256 + 32 j + l):
//  1. each warp ranks its keys in order: equal digits of one item are ranked with
//     __match_any_sync and counted into the warp's own row of digit counters (warp-level
//     sync only);
//  2. one pass over (digit, warp) turns the counters into the staging position of every
//     (digit, warp) run: digit starts (a scan over the digits), then the warps in order;
//  3. the keys are staged in shared memory in digit order and written out in that order:
//     a digit's keys go to consecutive global positions, so a warp writes runs.
__global__ void __launch_bounds__(kSortThreads, 4) k_sort_scatter(const unsigned long long* n_live, const unsigned int* kin,
                                                                  const unsigned int* iin, unsigned int* kout,
                                                                  unsigned int* iout, int shift,
                                                                  const unsigned int* offsets) {
  constexpr int kWarps = kSortThreads / 32, kIter = kSortThreads * kSortItems;
  __shared__ unsigned int s_off[256];                  // next global position of each digit
  __shared__ int s_delta[256];                         // global position - staged position
  __shared__ unsigned int s_wc[kWarps][256];           // per-warp digit counts, then run starts
  __shared__ unsigned int s_w[kWarps];
  __shared__ unsigned int s_k[kIter], s_i[kIter];
  const unsigned int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, t = threadIdx.x;
  s_off[t] = offsets[t * kSortBlocks + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s_wc[w][t] = 0;
  __syncthreads();
  const unsigned long long n = *n_live, c = sort_chunk(n);
  const unsigned long long b0 = blockIdx.x * c, b1 = b0 + c < n ? b0 + c : n;
  const unsigned int wbase = warp * (32u * kSortItems);
  unsigned int nk[kSortItems], ni[kSortItems];
  auto load = [&](unsigned long long base) {
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const unsigned long long i = base + wbase + 32u * j + lane;
      if (i < b1) {
        nk[j] = kin[i];
        ni[j] = iin[i];
      }
    }
  };
  if (b0 < b1) load(b0);
  for (unsigned long long base = b0; base < b1; base += kIter) {
    unsigned int k[kSortItems], ix[kSortItems], r[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      k[j] = nk[j];
      ix[j] = ni[j];
    }
    if (base + kIter < b1) load(base + kIter);
    const unsigned int m_it = (unsigned int)(b1 - base < (unsigned long long)kIter ? b1 - base : kIter);
    // 1. ranks inside the warp's run of each digit
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const bool valid = wbase + 32u * j + lane < m_it;
      const unsigned int d = valid ? (k[j] >> shift) & 255u : 256u + lane;   // invalid lanes match only themselves
      const unsigned int m = __match_any_sync(0xffffffffu, d);
      const unsigned int below = __popc(m & ((1u << lane) - 1u));
      if (valid) r[j] = s_wc[warp][d] + below;
      __syncwarp();
      if (valid && below == 0) s_wc[warp][d] += __popc(m);
      __syncwarp();
    }
    __syncthreads();
    // 2. staging starts: digit t's count over the warps, scanned over the digits
    unsigned int cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) cnt += s_wc[w][t];
    unsigned int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    unsigned int start = incl - cnt;
    for (unsigned int w = 0; w < warp; ++w) start += s_w[w];
    s_delta[t] = (int)s_off[t] - (int)start;
    s_off[t] += cnt;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {   // the runs of digit t, warp by warp
      const unsigned int v = s_wc[w][t];
      s_wc[w][t] = start;
      start += v;
    }
    __syncthreads();
    // 3. staged in digit order, then out
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      if (wbase + 32u * j + lane < m_it) {
        const unsigned int q = s_wc[warp][(k[j] >> shift) & 255u] + r[j];
        s_k[q] = k[j];
        s_i[q] = ix[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const unsigned int q = (unsigned int)(j * kSortThreads) + t;
      if (q < m_it) {
        const unsigned int kk = s_k[q];
        const unsigned int g = (unsigned int)((int)q + s_delta[(kk >> shift) & 255u]);
        kout[g] = kk;
        iout[g] = s_i[q];
      }
    }
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s_wc[w][t] = 0;
    __syncthreads();
  }
}

// up to kGroup arrays of one element size per launch: gathered through the sorted indices
// into the scratch (array j at tmp + j * cap), then copied back over the live elements
template <typename T>
struct SortGroup {
  T* a[kGroup];
  int na;
};

template <typename T>
__global__ void __launch_bounds__(kSortThreads) k_sort_gather(const unsigned long long* n_live, SortGroup<T> g,
                                                              T* tmp, unsigned long long cap, const unsigned int* idx) {
  const unsigned long long n = *n_live;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned int s = idx[i];
    T v[kGroup];
#pragma unroll
    for (int j = 0; j < kGroup; ++j)
      if (j < g.na) v[j] = g.a[j][s];
#pragma unroll
    for (int j = 0; j < kGroup; ++j)
      if (j < g.na) tmp[(unsigned long long)j * cap + i] = v[j];
  }
}

template <typename T>
__global__ void __launch_bounds__(kSortThreads) k_sort_copy(const unsigned long long* n_live, const T* tmp,
                                                            unsigned long long cap, SortGroup<T> g) {
  const unsigned long long n = *n_live;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    T v[kGroup];
#pragma unroll
    for (int j = 0; j < kGroup; ++j)
      if (j < g.na) v[j] = tmp[(unsigned long long)j * cap + i];
#pragma unroll
    for (int j = 0; j < kGroup; ++j)
      if (j < g.na) g.a[j][i] = v[j];
  }
}

}  // namespace qedk

using namespace qedk;

#define SFAIL(code, ...)     \
  do {                       \
    set_error(__VA_ARGS__);  \
    return code;             \
  } while (0)
#define SCK(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) SFAIL(QED_ERR_CUDA, "qed_sort_cells: %s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" qed_status qed_sort_cells(qed_ctx* c, qed_particles* set, const qed_fields* grid, void* stream) {
  const NvtxRange nvtx_range("qed_sort_cells");
  if (!c || !c->alive) SFAIL(QED_ERR_NOT_INITIALIZED, "qed_sort_cells: invalid context");
  if (!set || set->ctx != c) SFAIL(QED_ERR_INVALID_ARG, "qed_sort_cells: particle set missing or from another context");
  if (!grid || grid->kind != QED_FIELD_GRID2D) SFAIL(QED_ERR_INVALID_ARG, "qed_sort_cells: a grid field is needed");
  {
    const qed_status r = check_fields(grid, "qed_sort_cells");
    if (r != QED_OK) return r;
  }
  if (set->cap >= (1ull << 32)) SFAIL(QED_ERR_INVALID_ARG, "qed_sort_cells: capacity must be below 2^32");
  const unsigned long long tiles = (unsigned long long)((grid->nx + 31) / 32) * ((grid->ny + 31) / 32);
  if (tiles * 1024ull >= 0xFFFFFFFFull) SFAIL(QED_ERR_INVALID_ARG, "qed_sort_cells: grid too large for 32-bit keys");
  const unsigned int key_out = (unsigned int)(tiles * 1024ull);   // outside a bounded grid: last
  int bits = 1;
  while (bits < 32 && (1ull << bits) <= key_out) ++bits;
  const int passes = (bits + 7) / 8;
  // scratch: two (key, index) buffers, kGroup arrays of the largest element, the digit counts
  const size_t cap = set->cap ? set->cap : 1;
  const size_t need = 16 * cap + 8 * kGroup * cap + sizeof(unsigned int) * 256 * kSortBlocks;
  if (c->sort_bytes < need) {
    SCK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    if (c->sort_buf) cudaFree(c->sort_buf);
    c->sort_buf = nullptr;
    c->sort_bytes = 0;
    SCK(cudaMalloc(&c->sort_buf, need));
    c->sort_bytes = need;
  }
  unsigned char* b = static_cast<unsigned char*>(c->sort_buf);
  unsigned int* key[2] = {reinterpret_cast<unsigned int*>(b), reinterpret_cast<unsigned int*>(b + 4 * cap)};
  unsigned int* idx[2] = {reinterpret_cast<unsigned int*>(b + 8 * cap), reinterpret_cast<unsigned int*>(b + 12 * cap)};
  void* tmp = b + 16 * cap;
  unsigned int* counts = reinterpret_cast<unsigned int*>(b + (16 + 8 * kGroup) * cap);
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const unsigned long long* n_live = &c->st->n_live[set->species];
  int dev = 0, sms = 0;
  SCK(cudaGetDevice(&dev));
  SCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid_n = sms * 8;
  k_sort_keys<<<grid_n, kSortThreads, 0, s>>>(n_live, *grid, 1.0 / grid->dx, 1.0 / grid->dy,
                                               static_cast<const double*>(set->soa.x),
                                               static_cast<const double*>(set->soa.y), key[0], idx[0], key_out);
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    k_sort_hist<<<kSortBlocks, kSortThreads, 0, s>>>(n_live, key[cur], 8 * p, counts);
    k_sort_scan<<<1, 1024, 0, s>>>(counts);
    k_sort_scatter<<<kSortBlocks, kSortThreads, 0, s>>>(n_live, key[cur], idx[cur], key[cur ^ 1], idx[cur ^ 1], 8 * p,
                                                        counts);
    cur ^= 1;
  }
  const unsigned int* order = idx[cur];
  const size_t r = set->prec == QED_PREC_F64 ? 8 : 4;
  void* arr[12] = {set->soa.x, set->soa.y, set->soa.z, set->soa.px, set->soa.py, set->soa.pz, set->soa.s1,
                   set->soa.s2, set->soa.s3, set->soa.w, set->soa.id, set->soa.theta};
  const size_t esz[12] = {8, 8, 8, r, r, r, r, r, r, r, 8, r};
  const int na = set->species == QED_PHOTON ? 12 : 11;
  // groups of up to kGroup arrays of one element size: one gather and one copy each
  for (size_t size : {(size_t)8, (size_t)4}) {
    SortGroup<unsigned long long> g8{};
    SortGroup<unsigned int> g4{};
    int cnt = 0;
    for (int k = 0; k <= na; ++k) {
      const bool take = k < na && arr[k] && esz[k] == size;
      if (take) {
        if (size == 8) g8.a[cnt] = static_cast<unsigned long long*>(arr[k]);
        else g4.a[cnt] = static_cast<unsigned int*>(arr[k]);
        ++cnt;
      }
      if (cnt == kGroup || (k == na && cnt > 0)) {
        if (size == 8) {
          g8.na = cnt;
          k_sort_gather<unsigned long long><<<grid_n, kSortThreads, 0, s>>>(
              n_live, g8, static_cast<unsigned long long*>(tmp), cap, order);
          k_sort_copy<unsigned long long><<<grid_n, kSortThreads, 0, s>>>(
              n_live, static_cast<const unsigned long long*>(tmp), cap, g8);
        } else {
          g4.na = cnt;
          k_sort_gather<unsigned int><<<grid_n, kSortThreads, 0, s>>>(n_live, g4, static_cast<unsigned int*>(tmp),
                                                                     cap, order);
          k_sort_copy<unsigned int><<<grid_n, kSortThreads, 0, s>>>(n_live, static_cast<const unsigned int*>(tmp),
                                                                   cap, g4);
        }
        cnt = 0;
      }
    }
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) SFAIL(QED_ERR_CUDA, "qed_sort_cells: launch failed: %s", cudaGetErrorString(e));
  return QED_OK;
}
