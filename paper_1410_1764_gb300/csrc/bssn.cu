// BSSN stage kernel: the generated Einstein-equation right-hand side (Sec. 3.4
// and Sec. 5 name the system; the body comes from gen/systems.py) fused with
// Kreiss-Oliger dissipation and the Runge-Kutta update.
//
// One thread per point.  The FP64 pipe is the bound on GB300 (two FP64 FMA
// per clock per SM), so a block of 128 threads with up to 255 registers each
// and two blocks per SM already keeps it busy; neighbour values come through
// the read-only data cache.  A few block shapes are compiled; the autotuner
// picks one per system and grid.
#include "stage.cuh"
#include "generated/gen_bssn.cuh"
#include "generated/gen_bssn_x.cuh"
#include "generated/gen_bssn_xy.cuh"

namespace chemora {

template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) bssn_stage_kernel(Dims d, Scalars sc, StageParams a) {
  const int i = blockIdx.x * TX + threadIdx.x;
  const int j = blockIdx.y * TY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  Loader<24> ld{a.src + c, nullptr, d.sy, d.sz, d.sv};
  StageOut out{a, c, d.sv};
  chemora_bssn_point(ld, sc, out);
}

template <int TX, int TY, int MINB>
static int launch_bssn_variant(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, d.nz);
  bssn_stage_kernel<TX, TY, MINB><<<grid, dim3(TX, TY), 0, s>>>(d, sc, a);
  return launched("bssn_stage_kernel");
}

// x-sharing kernels: each warp is 32 consecutive x points of one row, and
// the x-direction first differences and the y/z derivative rows of the
// mixed xy/xz derivatives come from neighbouring lanes (the generated body
// chemora_bssn_x_point).  Used only when nx is a multiple of TX, so every lane
// is an interior point; rows beyond ny leave as whole warps.
template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) bssn_xstage_kernel(Dims d, Scalars sc, StageParams a) {
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

template <int TX, int TY, int MINB>
static int launch_bssn_xvariant(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  if (d.nx % TX != 0 || d.g < 3)
    return set_error(CHEMORA_EUNSUPPORTED, "x-sharing BSSN kernel needs nx %% %d == 0", TX);
  dim3 grid(d.nx / TX, (d.ny + TY - 1) / TY, d.nz);
  bssn_xstage_kernel<TX, TY, MINB><<<grid, dim3(TX, TY), 0, s>>>(d, sc, a);
  return launched("bssn_xstage_kernel");
}

// x- and y-sharing kernels: a block is 32 x TY points (TY >= 5); its
// prologue writes into shared memory, for every variable, the own first
// difference f(y+1) - f(y) and, for the 11 variables with second
// derivatives, the own raw z-derivative stencil -- plus the halo rows the
// stencils need (y differences at rows -3..-1 and TY, TY+1; z rows at -2, -1
// and TY, TY+1, computed by whole warps) -- then one barrier, then the
// generated body (chemora_bssn_xy_point) reads them.  Used only when nx % TX
// and ny % TY are 0, so every thread is an interior point and reaches the
// barrier.
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

template <int TX, int TY>
constexpr size_t xy_smem_bytes() {
  return (size_t)(24 * (TY + 5) + 11 * (TY + 4)) * TX * sizeof(double);
}

template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) bssn_xystage_kernel(Dims d, Scalars sc, StageParams a) {
  extern __shared__ double smem[];
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

template <int TX, int TY, int MINB>
static int launch_bssn_xyvariant(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  if (d.nx % TX != 0 || d.ny % TY != 0 || d.g < 3)
    return set_error(CHEMORA_EUNSUPPORTED, "xy-sharing BSSN kernel needs nx %% %d == ny %% %d == 0", TX, TY);
  constexpr size_t smem = xy_smem_bytes<TX, TY>();
  static bool attr_set = false;
  if (!attr_set) {
    CHEMORA_CUDA(cudaFuncSetAttribute(bssn_xystage_kernel<TX, TY, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  dim3 grid(d.nx / TX, d.ny / TY, d.nz);
  bssn_xystage_kernel<TX, TY, MINB><<<grid, dim3(TX, TY), smem, s>>>(d, sc, a);
  return launched("bssn_xystage_kernel");
}

// Launch shapes the autotuner chooses from (variant 0 is the default).
const LaunchVariant kBssnVariants[] = {
    {32, 4, 2, launch_bssn_variant<32, 4, 2>},
    {32, 2, 4, launch_bssn_variant<32, 2, 4>},
    {64, 2, 2, launch_bssn_variant<64, 2, 2>},
    {16, 8, 2, launch_bssn_variant<16, 8, 2>},
    {32, 8, 1, launch_bssn_variant<32, 8, 1>},
    {32, 4, 3, launch_bssn_variant<32, 4, 3>},
    {32, 4, 4, launch_bssn_variant<32, 4, 4>},
    {64, 2, 3, launch_bssn_variant<64, 2, 3>},
    {32, 2, 4, launch_bssn_xvariant<32, 2, 4>, 1},
    {32, 4, 2, launch_bssn_xvariant<32, 4, 2>, 1},
    {64, 2, 2, launch_bssn_xvariant<64, 2, 2>, 1},
    {32, 2, 5, launch_bssn_xvariant<32, 2, 5>, 1},
    {32, 2, 6, launch_bssn_xvariant<32, 2, 6>, 1},
    {32, 2, 8, launch_bssn_xvariant<32, 2, 8>, 1},
    {32, 8, 1, launch_bssn_xyvariant<32, 8, 1>, 2},
    {32, 8, 2, launch_bssn_xyvariant<32, 8, 2>, 2},
    {32, 16, 1, launch_bssn_xyvariant<32, 16, 1>, 2},
};
const int kNumBssnVariants = sizeof(kBssnVariants) / sizeof(kBssnVariants[0]);

int launch_bssn_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant) {
  if (variant < 0 || variant >= kNumBssnVariants) variant = 0;
  const LaunchVariant& v = kBssnVariants[variant];
  if (v.xshare && (d.nx % v.tx != 0 || d.g < 3 || (v.xshare == 2 && d.ny % v.ty != 0)))
    return kBssnVariants[0].launch(d, sc, a, s);
  return v.launch(d, sc, a, s);
}

}  // namespace chemora
