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
      case 1: {
        const double y = a.yn[cv];
        a.acc[cv] = fma(a.c1, k, y);
        a.dst[cv] = fma(a.c2, k, y);
      } break;
      case 2:
      case 3:
        a.acc[cv] = fma(a.c1, k, a.acc[cv]);
        a.dst[cv] = fma(a.c2, k, a.yn[cv]);
        break;
      default:
        a.dst[cv] = fma(a.c1, k, a.acc[cv]);
        break;
    }
  }
}

}  // namespace chemora
