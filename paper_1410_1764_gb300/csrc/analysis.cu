// Analysis kernels: BSSN constraints (Hamiltonian, momentum, Gamma
// constraint; generated from gen/systems.py) and the discrete energy of the
// scalar wave equation (the "Energy" calculation of Fig. 2), with a
// deterministic two-pass reduction.
#include <math.h>

#include "internal.h"
#include "stage.cuh"
#include "generated/gen_bssn_constraints.cuh"

namespace chemora {

constexpr int CTX = 32, CTY = 4;

__global__ void __launch_bounds__(CTX * CTY, 2) bssn_constraints_kernel(Dims d, Scalars sc,
                                                                        const double* __restrict__ st,
                                                                        double* __restrict__ out) {
  const int i = blockIdx.x * CTX + threadIdx.x;
  const int j = blockIdx.y * CTY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  Loader<24> ld{st + c, nullptr, d.sy, d.sz, d.sv};
  double o[7];
  ArrayOut<7> ao{o};
  chemora_bssn_constraints_point(ld, sc, ao);
#pragma unroll
  for (int q = 0; q < 7; ++q) out[c + q * d.sv] = o[q];
}

constexpr int EB = 256;  // threads per energy block

// Per-block partial sums of e = 1/2 (rho^2 - u Lap_h u) over the interior
// (x fastest linear order, a fixed tree inside the block).
__global__ void __launch_bounds__(EB) wave_energy_kernel(Dims d, double i12h2, const double* __restrict__ st,
                                                         double* __restrict__ partial, int64_t npts) {
  __shared__ double red[EB];
  double acc = 0.0;
  const int64_t plane = (int64_t)d.nx * d.ny;
  for (int64_t t = (int64_t)blockIdx.x * EB + threadIdx.x; t < npts; t += (int64_t)gridDim.x * EB) {
    const int k = (int)(t / plane);
    const int64_t r = t - (int64_t)k * plane;
    const int j = (int)(r / d.nx);
    const int i = (int)(r - (int64_t)j * d.nx);
    const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
    const double* u = st + c;
    const int64_t sv[3] = {1, d.sy, d.sz};
    double lap = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int64_t o = sv[q];
      const double f0 = u[0];
      const double d1 = (u[o] - f0) + (u[-o] - f0);
      const double d2 = (u[2 * o] - f0) + (u[-2 * o] - f0);
      lap += (16.0 * d1 - d2) * i12h2;
    }
    const double rho = st[d.sv + c];
    acc += 0.5 * (rho * rho - u[0] * lap);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = EB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int n, double scale, double* out) {
  __shared__ double red[EB];
  double acc = 0.0;
  for (int t = threadIdx.x; t < n; t += EB) acc += partial[t];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = EB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

}  // namespace chemora

using namespace chemora;

extern "C" {

int chemora_constraints(chemora_system* sys, const double* state, double* out, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (sys->kind != CHEMORA_BSSN) return set_error(CHEMORA_EINVAL, "chemora_constraints needs a CHEMORA_BSSN system");
  if (!state || !out) return set_error(CHEMORA_EINVAL, "NULL state or out");
  const Dims& d = sys->grid->d;
  dim3 grid((d.nx + CTX - 1) / CTX, (d.ny + CTY - 1) / CTY, d.nz);
  bssn_constraints_kernel<<<grid, dim3(CTX, CTY), 0, (cudaStream_t)stream>>>(d, sys->sc, state, out);
  return launched("bssn_constraints_kernel");
}

int chemora_energy(chemora_system* sys, const double* state, double* energy, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (sys->kind != CHEMORA_WAVE || sys->sc.order != 4)
    return set_error(CHEMORA_EINVAL, "chemora_energy needs a 4th-order CHEMORA_WAVE system");
  if (!state || !energy) return set_error(CHEMORA_EINVAL, "NULL state or energy");
  int rc = ensure_scratch(sys);  // partial sums live in the RK accumulator
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Dims& d = sys->grid->d;
  const int64_t npts = (int64_t)d.nx * d.ny * d.nz;
  int nblk = (int)((npts + EB - 1) / EB);
  if (nblk > 1024) nblk = 1024;
  double* partial = sys->scratch;
  double* dev_out = sys->scratch + nblk;
  wave_energy_kernel<<<nblk, EB, 0, s>>>(d, sys->sc.i12h2, state, partial, npts);
  if ((rc = launched("wave_energy_kernel"))) return rc;
  const double h = sys->grid->dx;
  sum_partials_kernel<<<1, EB, 0, s>>>(partial, nblk, h * h * h, dev_out);
  if ((rc = launched("sum_partials_kernel"))) return rc;
  CHEMORA_CUDA(cudaMemcpyAsync(energy, dev_out, sizeof(double), cudaMemcpyDeviceToHost, s));
  CHEMORA_CUDA(cudaStreamSynchronize(s));
  return CHEMORA_OK;
}

}  // extern "C"

namespace chemora {

// Count non-finite interior values of nv grid functions (NaN/Inf sentinel).
__global__ void count_nonfinite_kernel(Dims d, int nv, const double* __restrict__ st,
                                       unsigned long long* count) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 4 + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  unsigned int bad = 0;
  for (int v = 0; v < nv; ++v) bad += isfinite(st[c + v * d.sv]) ? 0u : 1u;
  if (bad) atomicAdd(count, (unsigned long long)bad);
}

}  // namespace chemora

extern "C" int chemora_check_finite(chemora_system* sys, const double* state, int64_t* nonfinite,
                                    void* stream) {
  using namespace chemora;
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (!state) return set_error(CHEMORA_EINVAL, "state is NULL");
  int rc = ensure_scratch(sys);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Dims& d = sys->grid->d;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(sys->scratch);
  CHEMORA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  dim3 grid((d.nx + 31) / 32, (d.ny + 3) / 4, d.nz);
  count_nonfinite_kernel<<<grid, dim3(32, 4), 0, s>>>(d, sys->nvars, state, cnt);
  if ((rc = launched("count_nonfinite_kernel"))) return rc;
  unsigned long long h = 0;
  CHEMORA_CUDA(cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, s));
  CHEMORA_CUDA(cudaStreamSynchronize(s));
  if (nonfinite) *nonfinite = (int64_t)h;
  if (h) return set_error(CHEMORA_ENONFINITE, "%llu non-finite interior values", h);
  return CHEMORA_OK;
}
