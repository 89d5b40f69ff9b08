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
#include "device_types.cuh"

// The value `own` holds on the lane m further along x; sources outside the
// warp come from the halo values `ext` (w per side, on lanes 0..2w-1).
// Every lane executes both shuffles.  (Global scope: called by generated
// point bodies.)
__device__ __forceinline__ double chemora_xshfl(double own, double ext, int m, int w) {
  const int lane = threadIdx.x & 31;
  const int src = lane + m;
  const double a = __shfl_sync(0xffffffffu, own, src & 31);
  const int esrc = src < 0 ? src + w : src - 32 + w;
  const double b = __shfl_sync(0xffffffffu, ext, esrc & 31);
  return (src >= 0 && src < 32) ? a : b;
}

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

// Loader of the x-sharing kernels: a warp holds 32 consecutive x points of
// one row.  Besides neighbour loads it computes the lane's halo values: the
// first difference f(x+1) - f(x) at x0-3..x0-1 (lanes 0-2) and x0+32,
// x0+33 (lanes 3-4), and the raw y / z first-derivative stencils at x0-2,
// x0-1 (lanes 0-1) and x0+32, x0+33 (lanes 2-3), x0 the warp's first x.
// Other lanes evaluate at their own point (unused, in bounds).  With the
// grid's nx a multiple of 32 and 3 ghost layers every access is in bounds.
template <int NV>
struct XLoader {
  const double* __restrict__ p;
  int64_t sy, sz, sv;
  int xo_dx, xo_d1;
  __device__ __forceinline__ double operator()(int v, int dx, int dy, int dz) const {
    return __ldg(p + v * sv + dx + dy * sy + dz * sz);
  }
  // one = 1.0, eight = 8.0 from the constant table: differences are
  // fma(b, -1, a), exact like a - b
  __device__ __forceinline__ double ext_dx(int v, double one) const {
    const double* q = p + v * sv + xo_dx;
    return fma(__ldg(q), -one, __ldg(q + 1));
  }
  __device__ __forceinline__ double ext_d1y(int v, double one, double eight) const {
    const double* q = p + v * sv + xo_d1;
    return d1_row(q, sy, one, eight);
  }
  __device__ __forceinline__ double ext_d1z(int v, double one, double eight) const {
    const double* q = p + v * sv + xo_d1;
    return d1_row(q, sz, one, eight);
  }
  // 8 (f(+1) - f(-1)) - (f(+2) - f(-2)) along stride s
  static __device__ __forceinline__ double d1_row(const double* q, int64_t s, double one, double eight) {
    const double p1 = fma(__ldg(q - s), -one, __ldg(q + s));
    const double p2 = fma(__ldg(q - 2 * s), -one, __ldg(q + 2 * s));
    return fma(eight, p1, -p2);
  }
};

// Output functors for the generated point bodies.
template <int NV>
struct ArrayOut {
  double (&a)[NV];
  __device__ __forceinline__ void operator()(int v, double x) const { a[v] = x; }
};

// Runge-Kutta update fused into the stage kernel, applied to one variable
// as soon as its right-hand side is known (shortens the outputs' live
// ranges).  The rounding follows the classic form
// y_{n+1} = y_n + dt/6 ((k1 + 2 k2) + 2 k3 + k4) and y_{s+1} = y_n + (c_s dt) k_s
// exactly (one rounding per add and multiply, no contraction): the states
// of near-flat BSSN data carry 1e-10 perturbations on O(1) backgrounds,
// where a one-ulp change of the update is a 2e-6 relative change of the
// perturbation.  Each add and multiply is an fma with an exact unit
// operand from the constant table (a + b = fma(a, 1, b), a b = fma(a, b, -0)):
// the same values, issued at the fma rate.
//   mode 0: dst = k
//   mode 1: acc = k;          dst = yn + c2 k
//   mode 2, 3: acc += 2 k;    dst = yn + c2 k   (2k exact: one rounding)
//   mode 4: dst = yn + c1 (acc + k)
struct StageOut {
  const StageParams& a;
  int64_t c, sv;
  double one, two, mzero;  // 1, 2, -0 from the constant table
  __device__ __forceinline__ void operator()(int v, double k) const {
    const int64_t cv = c + v * sv;
    switch (a.mode) {
      case 0:
        a.dst[cv] = k;
        break;
      case 1:
        a.acc[cv] = k;
        a.dst[cv] = __fma_rn(__fma_rn(a.c2, k, mzero), one, a.yn[cv]);
        break;
      case 2:
      case 3:
        a.acc[cv] = __fma_rn(two, k, a.acc[cv]);
        a.dst[cv] = __fma_rn(__fma_rn(a.c2, k, mzero), one, a.yn[cv]);
        break;
      default:
        a.dst[cv] = __fma_rn(__fma_rn(a.c1, __fma_rn(a.acc[cv], one, k), mzero), one, a.yn[cv]);
        break;
    }
  }
};
#define CHEMORA_STAGE_OUT(a, c, sv, sc) \
  StageOut { (a), (c), (sv), (sc).k[CHEMORA_K_ONE], (sc).k[CHEMORA_K_TWO], (sc).k[CHEMORA_K_MZERO] }

// The RK update of the scalar-wave systems, with the products contracted
// into the additions: dst = fma(c2, k, yn), acc = fma(2, k, acc),
// dst = fma(c1, acc + k, yn) -- one rounding fewer per update than the
// classic form and 1.75 instead of 2.75 FP64 instructions per variable and
// stage.  The wave solutions are O(1) with O(1) changes per step, so the
// contraction moves results by about an ulp per update, far inside the
// parity tolerance against the oracle (which rounds the classic form); the
// BSSN kernels keep StageOut, whose exact classic rounding the near-flat
// data need.  Every wave kernel uses this update, so the wave launch shapes and
// schedules stay bit-equal to each other.
struct StageOutFma {
  const StageParams& a;
  int64_t c, sv;
  double one, two;
  __device__ __forceinline__ void operator()(int v, double k) const {
    const int64_t cv = c + v * sv;
    switch (a.mode) {
      case 0:
        a.dst[cv] = k;
        break;
      case 1:
        a.acc[cv] = k;
        a.dst[cv] = __fma_rn(a.c2, k, a.yn[cv]);
        break;
      case 2:
      case 3:
        a.acc[cv] = __fma_rn(two, k, a.acc[cv]);
        a.dst[cv] = __fma_rn(a.c2, k, a.yn[cv]);
        break;
      default:
        a.dst[cv] = __fma_rn(a.c1, __fma_rn(a.acc[cv], one, k), a.yn[cv]);
        break;
    }
  }
};
#define CHEMORA_STAGE_OUT_FMA(a, c, sv, sc) \
  StageOutFma { (a), (c), (sv), (sc).k[CHEMORA_K_ONE], (sc).k[CHEMORA_K_TWO] }

}  // namespace chemora
