// Periodic ghost-zone fill (Sec. 2: the driver's ghost zones; on one GPU the
// "exchange" is the periodic image of the interior).
//
// One pass over the ghost points only: the six face slabs are enumerated as
// two z-slabs (full padded planes), two y-slabs (full padded rows of interior
// planes) and two x-slabs (the 2g edge points of interior rows).  Every
// ghost point copies the interior point with the same coordinates modulo the
// period, so edges and corners need no ordering between passes.  The kernel
// is memory-only (no FP64 arithmetic); z- and y-slab accesses are coalesced.
#include "internal.h"

namespace chemora {

__device__ __forceinline__ int wrap_idx(int i, int n, int g) {
  int r = (i - g) % n;
  return (r < 0 ? r + n : r) + g;
}

__global__ void ghost_fill_kernel(double* __restrict__ base, Dims d, int64_t total) {
  double* f = base + (int64_t)blockIdx.y * d.sv;
  const int g = d.g;
  const int64_t px = d.nx + 2 * g, py = d.ny + 2 * g;
  const int64_t zslab = 2 * g * py * px;
  const int64_t yslab = (int64_t)d.nz * 2 * g * px;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    if (t < zslab) {
      int64_t kk = t / (py * px), rem = t - kk * py * px;
      k = (int)(kk < g ? kk : kk + d.nz);
      j = (int)(rem / px);
      i = (int)(rem - (int64_t)j * px);
    } else if (t < zslab + yslab) {
      int64_t u = t - zslab;
      int64_t kk = u / (2 * g * px), rem = u - kk * 2 * g * px;
      k = (int)kk + g;
      int jj = (int)(rem / px);
      j = jj < g ? jj : jj + d.ny;
      i = (int)(rem - (int64_t)jj * px);
    } else {
      int64_t u = t - zslab - yslab;
      int64_t kk = u / ((int64_t)d.ny * 2 * g), rem = u - kk * d.ny * 2 * g;
      k = (int)kk + g;
      j = (int)(rem / (2 * g)) + g;
      int ii = (int)(rem % (2 * g));
      i = ii < g ? ii : ii + d.nx;
    }
    const int si = wrap_idx(i, d.nx, g), sj = wrap_idx(j, d.ny, g), sk = wrap_idx(k, d.nz, g);
    f[(int64_t)k * d.sz + (int64_t)j * d.sy + i] = f[(int64_t)sk * d.sz + (int64_t)sj * d.sy + si];
  }
}

// Periodic ghost fill restricted to the axes in `mask` (bit 0 x, 1 y, 2 z):
// a ghost point is copied from the point with its coordinates wrapped along
// the masked axes only; coordinates outside the interior along unmasked axes
// stay (those layers were filled by the caller, e.g. a halo exchange).
__global__ void ghost_fill_axes_kernel(double* __restrict__ base, Dims d, int mask) {
  double* f = base + (int64_t)blockIdx.y * d.sv;
  const int g = d.g;
  const int px = d.nx + 2 * g, py = d.ny + 2 * g, pz = d.nz + 2 * g;
  const int64_t total = (int64_t)px * py * pz;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % px), j = (int)((t / px) % py), k = (int)(t / ((int64_t)px * py));
    const int si = (mask & 1) ? wrap_idx(i, d.nx, g) : i;
    const int sj = (mask & 2) ? wrap_idx(j, d.ny, g) : j;
    const int sk = (mask & 4) ? wrap_idx(k, d.nz, g) : k;
    if (si == i && sj == j && sk == k) continue;
    f[(int64_t)k * d.sz + (int64_t)j * d.sy + i] = f[(int64_t)sk * d.sz + (int64_t)sj * d.sy + si];
  }
}

int fill_ghosts_axes(const Dims& d, int nvars, double* state, int mask, cudaStream_t s) {
  const int64_t total = (int64_t)(d.nx + 2 * d.g) * (d.ny + 2 * d.g) * (d.nz + 2 * d.g);
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  ghost_fill_axes_kernel<<<dim3((unsigned)blocks, (unsigned)nvars), 256, 0, s>>>(state, d, mask);
  return launched("ghost_fill_axes_kernel");
}

int64_t ghost_count(const Dims& d) {
  const int64_t g = d.g, px = d.nx + 2 * g, py = d.ny + 2 * g;
  return 2 * g * py * px + (int64_t)d.nz * 2 * g * px + (int64_t)d.nz * d.ny * 2 * g;
}

int fill_ghosts(const Dims& d, int nvars, double* state, cudaStream_t s) {
  const int64_t total = ghost_count(d);
  const int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  dim3 grid((unsigned)blocks, (unsigned)nvars);
  ghost_fill_kernel<<<grid, threads, 0, s>>>(state, d, total);
  return launched("ghost_fill_kernel");
}

}  // namespace chemora
