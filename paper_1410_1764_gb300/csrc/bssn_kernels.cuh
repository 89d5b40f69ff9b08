// Device bodies of the BSSN stage kernels: the generated Einstein-equation
// right-hand side (Sec. 3.4 and Sec. 5 name the system; the body comes from
// gen/systems.py) fused with Kreiss-Oliger dissipation and the Runge-Kutta
// update, one thread per point.
//
// Each body is a force-inlined function of the grid (Dims), the scalars (SC)
// and the stage arguments.  The ahead-of-time kernels in bssn.cu pass them as
// kernel parameters; the run-time specialised kernels (jit.cu) pass a Dims
// built from literals and an SC whose members are compile-time constants
// (Sec. 3.2.3: the run-time library compiles loop kernels once the parameter
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
  StageOut out = CHEMORA_STAGE_OUT(a, c, d.sv, sc);
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
  StageOut out = CHEMORA_STAGE_OUT(a, c, d.sv, sc);
  chemora_bssn_x_point(ld, sc, out);
}

// x and y sharing: a block is 32 x TY points (TY >= 5); its prologue writes
// into shared memory, for every variable, the own first difference
// f(y+1) - f(y) and, for the 11 variables with second derivatives, the own
// raw z-derivative stencil -- plus the halo rows the stencils need (y
// differences at rows -3..-1 and TY, TY+1; z rows at -2, -1 and TY, TY+1,
// computed by whole warps) -- then one barrier, then the generated body
// (chemora_bssn_xy_point) reads them.  Requires nx % TX == 0 (every lane an
// interior x point) and 3 ghost layers.  The last row of blocks may reach
// past ny: its rows beyond ny take part in the prologue and the barrier and
// then leave as whole warps; the prologue clamps the rows it reads to
// y <= ny + 1 (the highest row an interior point's stencils use, inside the
// ghost layers), so every access stays in the padded grid.
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
  const int y0 = blockIdx.y * TY;
  const int j = y0 + ty;
  const int k = blockIdx.z;
  // offset of point (i, y, k) for an interior-relative row y, clamped to
  // the rows the block's interior points read
  const int64_t base = (int64_t)(k + d.g) * d.sz + (i + d.g);
  auto at = [&](int y) { return base + (int64_t)((y < d.ny + 1 ? y : d.ny + 1) + d.g) * d.sy; };
  const double* src = a.src;
  const int64_t cj = at(j);
  const double one = sc.k[CHEMORA_K_ONE], eight = sc.k[CHEMORA_K_EIGHT];
  // own values
#pragma unroll 4
  for (int v = 0; v < 24; ++v) {
    const double* q = src + v * d.sv + cj;
    s_dy[(v * (TY + 5) + ty + 3) * TX + tx] = fma(__ldg(q), -one, __ldg(q + d.sy));
  }
#pragma unroll 1
  for (int vi = 0; vi < 11; ++vi) {
    const double* q = src + zrow_var(vi) * d.sv + cj;
    s_dz[(vi * (TY + 4) + ty + 2) * TX + tx] = XLoader<24>::d1_row(q, d.sz, one, eight);
  }
  // halo rows, one whole warp row each
  if (ty < 5) {
    const int row = ty < 3 ? ty : TY + ty;        // smem row; its y is y0 + row - 3
    const int64_t ch = at(y0 + row - 3);
#pragma unroll 4
    for (int v = 0; v < 24; ++v) {
      const double* q = src + v * d.sv + ch;
      s_dy[(v * (TY + 5) + row) * TX + tx] = fma(__ldg(q), -one, __ldg(q + d.sy));
    }
  }
  if (ty < 4) {
    const int row = ty < 2 ? ty : TY + ty;        // smem row; its y is y0 + row - 2
    const int64_t ch = at(y0 + row - 2);
#pragma unroll 1
    for (int vi = 0; vi < 11; ++vi) {
      const double* q = src + zrow_var(vi) * d.sv + ch;
      s_dz[(vi * (TY + 4) + row) * TX + tx] = XLoader<24>::d1_row(q, d.sz, one, eight);
    }
  }
  __syncthreads();
  if (j >= d.ny) return;  // whole warps (a warp is one row)
  const int lane = tx & 31;
  XYLoader<TX, TY> ld;
  ld.p = src + cj;
  ld.sy = d.sy;
  ld.sz = d.sz;
  ld.sv = d.sv;
  ld.xo_dx = lane < 3 ? -3 : (lane < 5 ? 29 : 0);
  ld.xo_d1 = lane < 2 ? -2 : (lane < 4 ? 30 : 0);
  ld.sdy_base = s_dy + (ty + 3) * TX + tx;
  ld.sdz_base = s_dz + (ty + 2) * TX + tx;
  StageOut out = CHEMORA_STAGE_OUT(a, cj, d.sv, sc);
  chemora_bssn_xy_point(ld, sc, out);
}

}  // namespace chemora
