/* A plain C caller of libchemora (no Python, no C++): the scalar wave of
 * Sec. 3 Eq. 1 on a 24 x 20 x 16 periodic grid, a plane wave advanced 20 RK4
 * steps through chemora_rk4_step on device memory the caller allocates, and
 * the same through chemora_rk4_step_host on a host buffer; prints the
 * largest difference between the two results and the discrete energy
 * before and after (chemora_energy).  Exit status 0 when every call
 * succeeded and the two results agree bit for bit. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "chemora.h"

#define CHECK(call)                                                          \
  do {                                                                       \
    int rc_ = (call);                                                        \
    if (rc_ != CHEMORA_OK) {                                                 \
      fprintf(stderr, "%s failed (%d): %s\n", #call, rc_, chemora_last_error()); \
      return 1;                                                              \
    }                                                                        \
  } while (0)

int main(void) {
  const int nx = 24, ny = 20, nz = 16, g = 2, nv = 2, steps = 20;
  const double h = 1.0 / nx, dt = 0.25 * h, pi = 3.14159265358979323846;
  chemora_grid* grid = NULL;
  chemora_system* sys = NULL;
  CHECK(chemora_grid_create(nx, ny, nz, nv, g, h, &grid));
  CHECK(chemora_system_create(grid, CHEMORA_WAVE, NULL, &sys));
  int64_t sy = 0, sz = 0, sv = 0;
  CHECK(chemora_grid_layout(grid, &sy, &sz, &sv));
  const size_t n = (size_t)nv * (size_t)sv;
  double* a = (double*)calloc(n, sizeof(double));
  double* b = (double*)calloc(n, sizeof(double));
  if (!a || !b) return 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t c = (size_t)(k + g) * sz + (size_t)(j + g) * sy + (i + g);
        a[c] = sin(2.0 * pi * (i * h + j * (1.0 / ny) + k * (1.0 / nz)));
      }
  memcpy(b, a, n * sizeof(double));
  double* d = NULL;
  if (cudaMalloc((void**)&d, n * sizeof(double)) != cudaSuccess) return 1;
  if (cudaMemcpy(d, a, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) return 1;
  double e0 = 0.0, e1 = 0.0;
  CHECK(chemora_fill_ghosts(sys, d, NULL));
  CHECK(chemora_energy(sys, d, &e0, NULL));
  CHECK(chemora_rk4_step(sys, d, dt, steps, NULL));
  CHECK(chemora_energy(sys, d, &e1, NULL));
  if (cudaMemcpy(a, d, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  CHECK(chemora_rk4_step_host(sys, b, dt, steps, NULL));
  double diff = 0.0;
  for (size_t q = 0; q < n; ++q) diff = fmax(diff, fabs(a[q] - b[q]));
  printf("max |device - host| = %.3e, energy %.17g -> %.17g\n", diff, e0, e1);
  cudaFree(d);
  free(a);
  free(b);
  chemora_destroy(sys);
  chemora_destroy(grid);
  return (diff == 0.0 && e1 <= e0 && e1 > 0.0) ? 0 : 2;
}
