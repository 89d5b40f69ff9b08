// Device bodies of the BSSN stage kernels: the generated Einstein-equation
// right-hand side (Sec. 3.4 and Sec. 5 name the system; the body comes from
// gen/systems.py) fused with Kreiss-Oliger dissipation and the Runge-Kutta
// update, one thread per point.
//
// Each body is a force-inlined function of the grid (Dims), the scalars (SC)
// and the stage arguments.  The ahead-of-time kernels in bssn.cu pass them as
// kernel parameters; the run-time specialised kernels (jit.cu) pass a Dims
// built from literals and an SC whose members are compile-time constants
// (Sec. 4.2.3: the run-time library compiles loop kernels once the parameter
// values are known, to cut code and register overhead),
// so strides, offsets and gauge switches fold into the instructions.  Only
// device code and device_types.cuh: the run-time compiler includes this file.
#pragma once
#include "stage.cuh"
#include "generated/gen_bssn.cuh"
#include "generated/gen_bssn_x.cuh"
#include "generated/gen_bssn_xy.cuh"

namespace chemora {

// One point per thread, neighbours through the read-only data cache.
template <int TX, int TY, class SC>
__device__ __forceinline__ void bssn_direct_body(const Dims& d, const SC& sc, const StageParams& a) {
  const int i = blockIdx.x * TX + threadIdx.x;
  const int j = blockIdx.y * TY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  Loader<24> ld{a.src + c, nullptr, d.sy, d.sz, d.sv};
  StageOut out{a, c, d.sv};
  chemora_bssn_point(ld, sc, out);
}

// x sharing: each warp is 32 consecutive x points of one row, and the
// x-direction first differences and the y/z derivative rows of the mixed
// xy/xz derivatives come from neighbouring lanes (the generated body
// chemora_bssn_x_point).  Requires nx % TX == 0, so every lane is an interior
// point; rows beyond ny leave as whole warps.
template <int TX, int TY, class SC>
__device__ __forceinline__ void bssn_x_body(const Dims& d, const SC& sc, const StageParams& a) {
  const int i = blockIdx.x * TX + threadIdx.x;
  const int j = blockIdx.y * TY + threadIdx.y;
  const int k = blockIdx.z;
  if (j >= d.ny) return;  // uniform over the warp
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  const int lane = threadIdx.x & 31;
  XLoader<24> ld{a.src + c, d.sy, d.sz, d.sv, lane < 3 ? -3 : (lane < 5 ? 29 : 0),
                 lane < 2 ? -2 : (lane < 4 ? 30 : 0)};
  StageOut out{a, c, d.sv};
  chemora_bssn_x_point(ld, sc, out);
}

// x and y sharing: a block is 32 x TY points (TY >= 5); its prologue writes
// into shared memory, for every variable, the own first difference
// f(y+1) - f(y) and, for the 11 variables with second derivatives, the own
// raw z-derivative stencil -- plus the halo rows the stencils need (y
// differences at rows -3..-1 and TY, TY+1; z rows at -2, -1 and TY, TY+1,
// computed by whole warps) -- then one barrier, then the generated body
// (chemora_bssn_xy_point) reads them.  Requires nx % TX == 0 and
// ny % TY == 0, so every thread is an interior point and reaches the barrier.
// z-row variables: phi, gt_ij (0-6) and alpha, beta^i (17-20)
__device__ __forceinline__ int zrow_var(int vi) { return vi < 7 ? vi : vi + 10; }

template <int TX, int TY>
struct XYLoader : XLoader<24> {
  const double* sdy_base;  // [24][TY + 5][TX] at this thread's (row + 3, lane)
  const double* sdz_base;  // [11][TY + 4][TX] at this thread's (row + 2, lane)
  __device__ __forceinline__ double sdy(int v, int m) const {
    return sdy_base[(v * (TY + 5) + m) * TX];
  }
  __device__ __forceinline__ double sdz(int vi, int m) const {
    return sdz_base[(vi * (TY + 4) + m) * TX];
  }
};

template <int TX, int TY, class SC>
__device__ __forceinline__ void bssn_xy_body(const Dims& d, const SC& sc, const StageParams& a,
                                             double* smem) {
  double* s_dy = smem;                          // [24][TY + 5][TX]
  double* s_dz = smem + 24 * (TY + 5) * TX;     // [11][TY + 4][TX]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * TX + tx;
  const int j = blockIdx.y * TY + ty;
  const int k = blockIdx.z;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  const double* src = a.src;
  // own values
#pragma unroll 4
  for (int v = 0; v < 24; ++v) {
    const double* q = src + v * d.sv + c;
    s_dy[(v * (TY + 5) + ty + 3) * TX + tx] = __ldg(q + d.sy) - __ldg(q);
  }
#pragma unroll 1
  for (int vi = 0; vi < 11; ++vi) {
    const double* q = src + zrow_var(vi) * d.sv + c;
    s_dz[(vi * (TY + 4) + ty + 2) * TX + tx] =
        8.0 * (__ldg(q + d.sz) - __ldg(q - d.sz)) - (__ldg(q + 2 * d.sz) - __ldg(q - 2 * d.sz));
  }
  // halo rows, one whole warp row each
  if (ty < 5) {
    const int row = ty < 3 ? ty : TY + ty;        // smem row
    const int64_t off = (int64_t)(row - 3 - ty) * d.sy;  // from the own row to that y
#pragma unroll 4
    for (int v = 0; v < 24; ++v) {
      const double* q = src + v * d.sv + c + off;
      s_dy[(v * (TY + 5) + row) * TX + tx] = __ldg(q + d.sy) - __ldg(q);
    }
  }
  if (ty < 4) {
    const int row = ty < 2 ? ty : TY + ty;
    const int64_t off = (int64_t)(row - 2 - ty) * d.sy;
#pragma unroll 1
    for (int vi = 0; vi < 11; ++vi) {
      const double* q = src + zrow_var(vi) * d.sv + c + off;
      s_dz[(vi * (TY + 4) + row) * TX + tx] =
          8.0 * (__ldg(q + d.sz) - __ldg(q - d.sz)) - (__ldg(q + 2 * d.sz) - __ldg(q - 2 * d.sz));
    }
  }
  __syncthreads();
  const int lane = tx & 31;
  XYLoader<TX, TY> ld;
  ld.p = src + c;
  ld.sy = d.sy;
  ld.sz = d.sz;
  ld.sv = d.sv;
  ld.xo_dx = lane < 3 ? -3 : (lane < 5 ? 29 : 0);
  ld.xo_d1 = lane < 2 ? -2 : (lane < 4 ? 30 : 0);
  ld.sdy_base = s_dy + (ty + 3) * TX + tx;
  ld.sdz_base = s_dz + (ty + 2) * TX + tx;
  StageOut out{a, c, d.sv};
  chemora_bssn_xy_point(ld, sc, out);
}

}  // namespace chemora
