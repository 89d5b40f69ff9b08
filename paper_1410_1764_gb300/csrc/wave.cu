// Scalar wave (Sec. 3, Eq. 1, two-variable form) and variable-speed wave
// stage kernels.  Bodies generated from gen/systems.py; a few block shapes
// are compiled for the autotuner.
#include "internal.h"
#include "stage.cuh"
#include "generated/gen_wave.cuh"
#include "generated/gen_wave_varc.cuh"

namespace chemora {

template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) wave_stage_kernel(Dims d, Scalars sc, StageParams a) {
  const int i = blockIdx.x * TX + threadIdx.x;
  const int j = blockIdx.y * TY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  Loader<2> ld{a.src + c, nullptr, d.sy, d.sz, d.sv};
  StageOut out = CHEMORA_STAGE_OUT(a, c, d.sv, sc);
  chemora_wave_point(ld, sc, out);
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) varc_stage_kernel(Dims d, Scalars sc, StageParams a) {
  const int i = blockIdx.x * TX + threadIdx.x;
  const int j = blockIdx.y * TY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  Loader<2> ld{a.src + c, a.coef + c, d.sy, d.sz, d.sv};
  StageOut out = CHEMORA_STAGE_OUT(a, c, d.sv, sc);
  chemora_varc_point(ld, sc, out);
}

template <int TX, int TY>
static int launch_wave_variant(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, d.nz);
  wave_stage_kernel<TX, TY><<<grid, dim3(TX, TY), 0, s>>>(d, sc, a);
  return launched("wave_stage_kernel");
}

template <int TX, int TY>
static int launch_varc_variant(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, d.nz);
  varc_stage_kernel<TX, TY><<<grid, dim3(TX, TY), 0, s>>>(d, sc, a);
  return launched("varc_stage_kernel");
}

const LaunchVariant kWaveVariants[] = {
    {32, 8, 0, launch_wave_variant<32, 8>},  {32, 4, 0, launch_wave_variant<32, 4>},
    {64, 4, 0, launch_wave_variant<64, 4>},  {128, 2, 0, launch_wave_variant<128, 2>},
    {32, 16, 0, launch_wave_variant<32, 16>}, {16, 16, 0, launch_wave_variant<16, 16>},
};
const int kNumWaveVariants = sizeof(kWaveVariants) / sizeof(kWaveVariants[0]);

const LaunchVariant kVarcVariants[] = {
    {32, 8, 0, launch_varc_variant<32, 8>},  {32, 4, 0, launch_varc_variant<32, 4>},
    {64, 4, 0, launch_varc_variant<64, 4>},  {128, 2, 0, launch_varc_variant<128, 2>},
    {32, 16, 0, launch_varc_variant<32, 16>}, {16, 16, 0, launch_varc_variant<16, 16>},
};
const int kNumVarcVariants = sizeof(kVarcVariants) / sizeof(kVarcVariants[0]);

int launch_wave_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant) {
  if (sc.order != 4) return launch_wave_order_stage(d, sc, a, s, variant);
  if (variant < 0 || variant >= kNumWaveVariants) variant = 0;
  return kWaveVariants[variant].launch(d, sc, a, s);
}

int launch_varc_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant) {
  if (variant < 0 || variant >= kNumVarcVariants) variant = 0;
  return kVarcVariants[variant].launch(d, sc, a, s);
}

}  // namespace chemora
