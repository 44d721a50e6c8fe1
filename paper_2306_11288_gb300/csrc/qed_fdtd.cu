// qed_fdtd.cu -- the 2D3V Yee field solver around the step (paper Sec. II B, z squeezed):
// the two curl equations in normalised units (c = 1),
//   Faraday: B -= dt curl E,   Ampere: E += dt (curl B - J),
// on the staggering Ex(i+1/2,j) Ey(i,j+1/2) Ez(i,j) Bx(i,j+1/2) By(i+1/2,j) Bz(i+1/2,j+1/2),
// currents on the E positions.  Gauss's law is not solved: the charge-conserving current
// deposition keeps it (Sec. II B).  Neighbours outside the grid are zero, or wrap.
//
// One thread per cell, the x index along the warp (coalesced rows of every array); each
// update reads the other field's two or three neighbours from L1/L2 and its own three
// components, and writes its three components: an HBM-bound stencil.  The updates are in
// place (Faraday reads only E, Ampere only B and J), and Ampere clears J behind it.
#include <cmath>

#include "qed_common.cuh"
#include "qed_internal.h"

namespace qedk {

__device__ __forceinline__ int fd_wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// value at (i, j) with i, j at most one cell outside the grid
__device__ __forceinline__ float fd_at(const float* a, int nx, int ny, int per, int i, int j) {
  if (per) {
    i = fd_wrap(i, nx);
    j = fd_wrap(j, ny);
  } else if (i < 0 || i >= nx || j < 0 || j >= ny) {
    return 0.0f;
  }
  return __ldg(a + (size_t)j * nx + i);
}

__global__ void __launch_bounds__(256) k_fdtd_b(qed_grid2d g, float cdx, float cdy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const int nx = g.nx, ny = g.ny, per = g.periodic;
  const size_t k = (size_t)j * nx + i;
  const float ez = g.Ez[k];
  const float ez_j1 = fd_at(g.Ez, nx, ny, per, i, j + 1), ez_i1 = fd_at(g.Ez, nx, ny, per, i + 1, j);
  const float ey = g.Ey[k], ey_i1 = fd_at(g.Ey, nx, ny, per, i + 1, j);
  const float ex = g.Ex[k], ex_j1 = fd_at(g.Ex, nx, ny, per, i, j + 1);
  // Bx(i,j+1/2): -dEz/dy;  By(i+1/2,j): +dEz/dx;  Bz(i+1/2,j+1/2): -(dEy/dx - dEx/dy)
  g.Bx[k] -= cdy * (ez_j1 - ez);
  g.By[k] += cdx * (ez_i1 - ez);
  g.Bz[k] -= cdx * (ey_i1 - ey) - cdy * (ex_j1 - ex);
}

__global__ void __launch_bounds__(256) k_fdtd_e(qed_grid2d g, float cdx, float cdy, float cdt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const int nx = g.nx, ny = g.ny, per = g.periodic;
  const size_t k = (size_t)j * nx + i;
  const float bz = g.Bz[k], bz_j0 = fd_at(g.Bz, nx, ny, per, i, j - 1), bz_i0 = fd_at(g.Bz, nx, ny, per, i - 1, j);
  const float by = g.By[k], by_i0 = fd_at(g.By, nx, ny, per, i - 1, j);
  const float bx = g.Bx[k], bx_j0 = fd_at(g.Bx, nx, ny, per, i, j - 1);
  // Ex(i+1/2,j): dBz/dy - Jx;  Ey(i,j+1/2): -dBz/dx - Jy;  Ez(i,j): dBy/dx - dBx/dy - Jz
  g.Ex[k] += cdy * (bz - bz_j0) - cdt * g.Jx[k];
  g.Ey[k] += -cdx * (bz - bz_i0) - cdt * g.Jy[k];
  g.Ez[k] += cdx * (by - by_i0) - cdy * (bx - bx_j0) - cdt * g.Jz[k];
  g.Jx[k] = 0.0f;
  g.Jy[k] = 0.0f;
  g.Jz[k] = 0.0f;
}

}  // namespace qedk

using namespace qedk;

extern "C" qed_status qed_fdtd_advance(const qed_grid2d* g, int which, double dt, void* stream) {
  const qedk::NvtxRange nvtx_range("qed_fdtd_advance");
  if (!g) {
    set_error("qed_fdtd_advance: grid is NULL");
    return QED_ERR_INVALID_ARG;
  }
  if (!g->Ex || !g->Ey || !g->Ez || !g->Bx || !g->By || !g->Bz || !g->Jx || !g->Jy || !g->Jz) {
    set_error("qed_fdtd_advance: grid arrays must be non-NULL");
    return QED_ERR_INVALID_ARG;
  }
  if (g->nx < 2 || g->ny < 2 || g->ny > 65535 || !(g->dx > 0.0) || !(g->dy > 0.0) || !std::isfinite(g->dx) ||
      !std::isfinite(g->dy) || (g->periodic != 0 && g->periodic != 1)) {
    set_error("qed_fdtd_advance: bad grid geometry");
    return QED_ERR_INVALID_ARG;
  }
  if (!(dt > 0.0) || !std::isfinite(dt)) {
    set_error("qed_fdtd_advance: dt must be positive and finite");
    return QED_ERR_INVALID_ARG;
  }
  if (which != QED_FDTD_B && which != QED_FDTD_E) {
    set_error("qed_fdtd_advance: which must be QED_FDTD_B or QED_FDTD_E");
    return QED_ERR_INVALID_ARG;
  }
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const dim3 grid((unsigned)((g->nx + 255) / 256), (unsigned)g->ny);
  const float cdx = (float)(dt / g->dx), cdy = (float)(dt / g->dy);
  if (which == QED_FDTD_B) k_fdtd_b<<<grid, 256, 0, s>>>(*g, cdx, cdy);
  else k_fdtd_e<<<grid, 256, 0, s>>>(*g, cdx, cdy, (float)dt);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("qed_fdtd_advance: launch failed: %s", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  return QED_OK;
}
