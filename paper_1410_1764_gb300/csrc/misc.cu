// Coefficient upload for the variable-speed wave, handle destruction, and the
// FP64 throughput probe used as the roofline's compute peak.
#include <math.h>

#include "internal.h"

namespace chemora {

__global__ void square_interior_kernel(const double* __restrict__ c, double* __restrict__ s, Dims d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx) return;
  const int64_t p = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  const double v = c[p];
  s[p] = v * v;
}

// Independent FMA chains: 8 per thread, enough to cover the FP64 latency.
__global__ void fp64_fma_probe_kernel(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-3 + q;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  if (s == 1234.5678) out[0] = s;  // keeps the chains live; never true
}

void destroy_batch(chemora_batch* b);
void destroy_amr(chemora_amr* A);

}  // namespace chemora

using namespace chemora;

extern "C" {

int chemora_system_set_speed(chemora_system* sys, const double* c, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (sys->kind != CHEMORA_WAVE_VARC)
    return set_error(CHEMORA_EINVAL, "chemora_system_set_speed needs a CHEMORA_WAVE_VARC system");
  if (!c) return set_error(CHEMORA_EINVAL, "c is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const Dims& d = sys->grid->d;
  const size_t fs = sys->grid->fsize;
  if (!sys->coef) {
    cudaError_t e = cudaMalloc(&sys->coef, 4 * fs * sizeof(double));  // s, D_x s, D_y s, D_z s
    if (e != cudaSuccess) {
      sys->coef = nullptr;
      cudaGetLastError();
      return set_error(CHEMORA_ENOMEM, "coefficient storage: %s", cudaGetErrorString(e));
    }
  }
  dim3 grid((d.nx + 127) / 128, d.ny, d.nz);
  square_interior_kernel<<<grid, 128, 0, s>>>(c, sys->coef, d);
  int rc = launched("square_interior_kernel");
  if (rc) return rc;
  if ((rc = fill_ghosts(d, 1, sys->coef, s))) return rc;
  // the speed is constant in time: its derivatives are taken once, here
  if ((rc = launch_varc_grad(d, sys->sc.i12h, sys->coef, sys->coef + fs, s))) return rc;
  if ((rc = fill_ghosts(d, 3, sys->coef + fs, s))) return rc;
  CHEMORA_CUDA(cudaStreamSynchronize(s));
  return CHEMORA_OK;
}

int chemora_fp64_peak(double* flops_per_s, void* stream) {
  if (!flops_per_s) return set_error(CHEMORA_EINVAL, "NULL output");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  CHEMORA_CUDA(cudaGetDevice(&dev));
  CHEMORA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* buf = nullptr;
  CHEMORA_CUDA(cudaMalloc(&buf, 64));
  cudaEvent_t e0, e1;
  CHEMORA_CUDA(cudaEventCreate(&e0));
  CHEMORA_CUDA(cudaEventCreate(&e1));
  const int blocks = sms * 2, threads = 256, iters = 4096;
  fp64_fma_probe_kernel<<<blocks, threads, 0, s>>>(buf, 64, 0.999, 1e-3);
  int rc = launched("fp64_fma_probe_kernel");
  float best = 1e30f;
  for (int rep = 0; rep < 5 && rc == CHEMORA_OK; ++rep) {
    cudaEventRecord(e0, s);
    fp64_fma_probe_kernel<<<blocks, threads, 0, s>>>(buf, iters, 0.999, 1e-3);
    rc = launched("fp64_fma_probe_kernel");
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc) return rc;
  *flops_per_s = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3);
  return CHEMORA_OK;
}

void chemora_destroy(void* handle) {
  if (!handle) return;
  if (is_handle(handle, H_GRID)) {
    chemora_grid* g = (chemora_grid*)handle;
    g->type = 0;
    delete g;
  } else if (is_handle(handle, H_SYSTEM)) {
    chemora_system* s = (chemora_system*)handle;
    free_step_graph(s);
    jit_free(s);
    chain_free(s);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->scratch) cudaFree(s->scratch);
    if (s->coef) cudaFree(s->coef);
    if (s->dev_state) cudaFree(s->dev_state);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    s->type = 0;
    delete s;
  } else if (is_handle(handle, H_BATCH)) {
    destroy_batch((chemora_batch*)handle);
  } else if (is_handle(handle, H_AMR)) {
    destroy_amr((chemora_amr*)handle);
  }
}

}  // extern "C"
