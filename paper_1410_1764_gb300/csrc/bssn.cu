// Ahead-of-time BSSN stage kernels: the device bodies of bssn_kernels.cuh
// compiled for a few launch shapes with the grid and scalars as kernel
// parameters; the autotuner picks one shape per system and grid.
//
// The FP64 pipe is the bound on GB300 (two FP64 FMA per clock per SM), so
// blocks of 64-256 threads with up to 255 registers each and a few blocks per
// SM already keep it busy.
#include <atomic>

#include "internal.h"
#include "bssn_kernels.cuh"

namespace chemora {

template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) bssn_stage_kernel(Dims d, Scalars sc, StageParams a) {
  bssn_direct_body<TX, TY>(d, sc, a);
}

template <int TX, int TY, int MINB>
static int launch_bssn_variant(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, d.nz);
  bssn_stage_kernel<TX, TY, MINB><<<grid, dim3(TX, TY), 0, s>>>(d, sc, a);
  return launched("bssn_stage_kernel");
}

template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) bssn_xstage_kernel(Dims d, Scalars sc, StageParams a) {
  bssn_x_body<TX, TY>(d, sc, a);
}

template <int TX, int TY, int MINB>
static int launch_bssn_xvariant(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  if (d.nx % TX != 0 || d.g < 3)
    return set_error(CHEMORA_EUNSUPPORTED, "x-sharing BSSN kernel needs nx %% %d == 0", TX);
  dim3 grid(d.nx / TX, (d.ny + TY - 1) / TY, d.nz);
  bssn_xstage_kernel<TX, TY, MINB><<<grid, dim3(TX, TY), 0, s>>>(d, sc, a);
  return launched("bssn_xstage_kernel");
}

template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) bssn_xystage_kernel(Dims d, Scalars sc, StageParams a) {
  extern __shared__ double smem[];
  bssn_xy_body<TX, TY>(d, sc, a, smem);
}

template <int TX, int TY, int MINB>
static int launch_bssn_xyvariant(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  if (d.nx % TX != 0 || d.g < 3)
    return set_error(CHEMORA_EUNSUPPORTED, "xy-sharing BSSN kernel needs nx %% %d == 0", TX);
  constexpr unsigned smem = bssn_xy_smem_bytes(TX, TY);
  // the dynamic shared-memory limit is a per-device function attribute: set
  // once per device (a bit per device ordinal; thread-safe)
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  CHEMORA_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_set.load() & bit)) {
    CHEMORA_CUDA(cudaFuncSetAttribute(bssn_xystage_kernel<TX, TY, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set.fetch_or(bit);
  }
  dim3 grid(d.nx / TX, (d.ny + TY - 1) / TY, d.nz);
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
    // fewer rows per block: more registers per thread (168-200), fewer warps
    {32, 5, 2, launch_bssn_xyvariant<32, 5, 2>, 2},
    {32, 6, 2, launch_bssn_xyvariant<32, 6, 2>, 2},
    {32, 7, 2, launch_bssn_xyvariant<32, 7, 2>, 2},
    {32, 12, 1, launch_bssn_xyvariant<32, 12, 1>, 2},
};
const int kNumBssnVariants = sizeof(kBssnVariants) / sizeof(kBssnVariants[0]);

int launch_bssn_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant) {
  if (variant < 0 || variant >= kNumBssnVariants) variant = 0;
  const LaunchVariant& v = kBssnVariants[variant];
  if (v.xshare && (d.nx % v.tx != 0 || d.g < 3))
    return kBssnVariants[0].launch(d, sc, a, s);
  return v.launch(d, sc, a, s);
}

}  // namespace chemora
