// Fused stage kernel template: stencils + right-hand side + Runge-Kutta
// update for one interior point per thread (Sec. 3.2: the generated "RHS"
// calculation fused with the time integrator's update, Sec. 2).
//
// The point bodies are generated (csrc/generated/gen_*.cuh) from symbolic
// equation lists; they read neighbour values through the loader `ld(v, dx,
// dy, dz)`, whose offsets are compile-time constants after inlining.  All
// derivatives of a point live in registers; nothing but the state and the
// Runge-Kutta buffers touches global memory.  FP64 throughput, not memory,
// bounds these kernels on GB300, so one thread per point with read-only
// cached neighbour loads keeps the FP64 pipe fed with few warps per SM.
#pragma once
#include "internal.h"

namespace chemora {

template <int NV>
struct Loader {
  const double* __restrict__ p;  // centre point of variable 0
  const double* __restrict__ q;  // centre point of the coefficient field
  int64_t sy, sz, sv;
  __device__ __forceinline__ double operator()(int v, int dx, int dy, int dz) const {
    const int64_t off = dx + dy * sy + dz * sz;
    if (v < NV) return __ldg(p + v * sv + off);
    return __ldg(q + off);
  }
};

// Runge-Kutta update fused into the stage kernel.  The rounding follows the
// classic form y_{n+1} = y_n + dt/6 ((k1 + 2 k2) + 2 k3 + k4) and
// y_{s+1} = y_n + (c_s dt) k_s exactly (explicit round-to-nearest operations,
// no contraction): the states of near-flat BSSN data carry 1e-10
// perturbations on O(1) backgrounds, where a one-ulp change of the update is
// a 2e-6 relative change of the perturbation.
//   mode 0: dst = k
//   mode 1: acc = k;          dst = yn + c2 k
//   mode 2, 3: acc += 2 k;    dst = yn + c2 k
//   mode 4: dst = yn + c1 (acc + k)
template <int NV>
__device__ __forceinline__ void stage_epilogue(const double (&out)[NV], int64_t c, int64_t sv,
                                               const StageParams& a) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int64_t cv = c + v * sv;
    const double k = out[v];
    switch (a.mode) {
      case 0:
        a.dst[cv] = k;
        break;
      case 1:
        a.acc[cv] = k;
        a.dst[cv] = __dadd_rn(a.yn[cv], __dmul_rn(a.c2, k));
        break;
      case 2:
      case 3:
        a.acc[cv] = fma(2.0, k, a.acc[cv]);  // 2k is exact: one rounding, as acc + 2k
        a.dst[cv] = __dadd_rn(a.yn[cv], __dmul_rn(a.c2, k));
        break;
      default:
        a.dst[cv] = __dadd_rn(a.yn[cv], __dmul_rn(a.c1, __dadd_rn(a.acc[cv], k)));
        break;
    }
  }
}

}  // namespace chemora
