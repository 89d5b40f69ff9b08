// RK4 steps without any device allocation, for callers that cannot allocate.
//
// Who needs this: code that runs where cudaMalloc is unavailable or
// forbidden -- inside a host callback or an allocator hook, in a process
// whose device memory is carved up by a framework that must see every
// allocation, or in a real-time loop that may not risk an allocation's
// implicit synchronisation or failure part-way through a run.
// chemora_rk4_step allocates its three work states on first use;
// chemora_rk4_step_noalloc instead uses one fixed scratch array compiled into
// the library.
//
// The scratch is a file-scope __device__ array of CHEMORA_NOALLOC_SCRATCH_DOUBLES
// doubles (32 MiB).  Host code cannot use the array's name as a device
// address (on the host it names a stand-in object), so the device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on the device.  With CUDA's lazy module
// loading that lookup is also what loads this file's module and reserves the
// 32 MiB on the device (held until the process exits), so the first call can
// fail for lack of device memory (reported as CHEMORA_ENOMEM); it should come
// before any stream capture.  All calls share the one array: calls whose work
// overlaps on the GPU (different streams, or different host threads) race
// on it and must be serialised by the caller.  The array keeps whatever the
// last call left in it; this entry point never reads an element it has not
// written earlier in the same call (the accumulator and stage states are
// written before they are read, ghost zones are filled before stencils read
// them), so nothing needs clearing.
#include <math.h>

#include <mutex>

#include "internal.h"

#define CHEMORA_NOALLOC_SCRATCH_DOUBLES 4194304LL  // three states of up to 1,398,101 doubles

namespace chemora {

static __device__ __align__(256) double g_noalloc_scratch[CHEMORA_NOALLOC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
static double* g_noalloc_addr[kMaxDevices];
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (set-up on the
// first call per device).
static int noalloc_scratch(double** out) {
  int dev = 0;
  CHEMORA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(CHEMORA_EUNSUPPORTED, "device ordinal %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e == cudaErrorMemoryAllocation) {
      (void)cudaGetLastError();
      return set_error(CHEMORA_ENOMEM,
                       "chemora_rk4_step_noalloc: no room for the %lld-byte static scratch on device %d",
                       (long long)(CHEMORA_NOALLOC_SCRATCH_DOUBLES * 8), dev);
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return CHEMORA_OK;
}

}  // namespace chemora

using namespace chemora;

extern "C" int chemora_rk4_step_noalloc(chemora_system* sys, double* state, double dt, int nsteps,
                                        void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (!state) return set_error(CHEMORA_EINVAL, "state is NULL");
  if (nsteps < 0) return set_error(CHEMORA_EINVAL, "nsteps < 0");
  if (!isfinite(dt)) return set_error(CHEMORA_EINVAL, "dt not finite");
  if (sys->kind == CHEMORA_WAVE_VARC && !sys->coef)
    return set_error(CHEMORA_EINVAL, "variable-speed system without a speed (chemora_system_set_speed)");
  const int64_t n = (int64_t)sys->nvars * sys->grid->fsize;
  if (3 * n > CHEMORA_NOALLOC_SCRATCH_DOUBLES)
    return set_error(CHEMORA_EINVAL,
                     "chemora_rk4_step_noalloc: a state of %lld doubles needs %lld scratch doubles; "
                     "the static scratch holds %lld (nvars*(nx+2g)*(ny+2g)*(nz+2g) <= %lld)",
                     (long long)n, (long long)(3 * n), (long long)CHEMORA_NOALLOC_SCRATCH_DOUBLES,
                     (long long)(CHEMORA_NOALLOC_SCRATCH_DOUBLES / 3));
  double* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Dims& d = sys->grid->d;
  const int nv = sys->nvars;
  double* A = base;
  double* Sa = base + n;
  double* Sb = base + 2 * n;
  for (int step = 0; step < nsteps; ++step) {
    StageParams p{};
    p.coef = sys->coef;
    if ((rc = fill_ghosts(d, nv, state, s))) return rc;
    p.src = state; p.yn = state; p.acc = A; p.dst = Sa; p.c2 = 0.5 * dt; p.mode = 1;
    if ((rc = launch_stage(sys->kind, d, sys->sc, p, s))) return rc;
    if ((rc = fill_ghosts(d, nv, Sa, s))) return rc;
    p.src = Sa; p.dst = Sb; p.c2 = 0.5 * dt; p.mode = 2;
    if ((rc = launch_stage(sys->kind, d, sys->sc, p, s))) return rc;
    if ((rc = fill_ghosts(d, nv, Sb, s))) return rc;
    p.src = Sb; p.dst = Sa; p.c2 = dt; p.mode = 3;
    if ((rc = launch_stage(sys->kind, d, sys->sc, p, s))) return rc;
    if ((rc = fill_ghosts(d, nv, Sa, s))) return rc;
    p.src = Sa; p.dst = state; p.c1 = dt / 6.0; p.c2 = 0.0; p.mode = 4;
    if ((rc = launch_stage(sys->kind, d, sys->sc, p, s))) return rc;
  }
  return fill_ghosts(d, nv, state, s);
}
