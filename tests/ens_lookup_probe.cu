// Test helper (not part of the library): a tile's ensemble by the streaming passes' warp-ballot
// lookup (find_ens_warp) and by the per-thread binary search (find_ens), for a list of tiles,
// so that a test can check the two agree on every tile of any offset table.
#include <cstdint>
#include "../paper_2306_11288_gb300/csrc/qed_kernels.cuh"

// one warp per query: every lane calls find_ens_warp with the warp's tile; lane 0 stores it
// and find_ens's answer for the same tile
__global__ void k_ens_lookup(const unsigned int* off, int n, const unsigned int* g, int nq, int* warp_ans,
                             int* search_ans) {
  const int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (q >= nq) return;   // whole warps leave together (blockDim is a multiple of 32)
  const int w = qedk::find_ens_warp(off, n, g[q]);
  if ((threadIdx.x & 31u) == 0u) {
    warp_ans[q] = w;
    search_ans[q] = qedk::find_ens(off, n, g[q]);
  }
}

// off: device array of n + 1 non-decreasing offsets with off[0] = 0 (1 <= n <= 1024);
// g: nq tiles, each below off[n]; answers: two device arrays of nq ints.  Returns a
// cudaError_t value; 1 for bad sizes.
extern "C" int ens_lookup_eval(const unsigned int* off, int n, const unsigned int* g, int nq, int* warp_ans,
                               int* search_ans) {
  if (n < 1 || n > 1024 || nq < 0) return 1;
  if (nq == 0) return 0;
  const long long threads = 32LL * nq;
  k_ens_lookup<<<(unsigned int)((threads + 255) / 256), 256>>>(off, n, g, nq, warp_ans, search_ans);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  return (int)cudaDeviceSynchronize();
}
