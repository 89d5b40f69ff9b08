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
};
const int kNumBssnVariants = sizeof(kBssnVariants) / sizeof(kBssnVariants[0]);

int launch_bssn_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant) {
  if (variant < 0 || variant >= kNumBssnVariants) variant = 0;
  const LaunchVariant& v = kBssnVariants[variant];
  if (v.xshare && (d.nx % v.tx != 0 || d.g < 3)) return kBssnVariants[0].launch(d, sc, a, s);
  return v.launch(d, sc, a, s);
}

}  // namespace chemora
