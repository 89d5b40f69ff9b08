// Scalar wave (Sec. 3, Eq. 1, two-variable form) and variable-speed wave
// stage kernels.  Bodies generated from gen/systems.py.
#include "stage.cuh"
#include "generated/gen_wave.cuh"
#include "generated/gen_wave_varc.cuh"

namespace chemora {

constexpr int WTX = 32, WTY = 8;

__global__ void __launch_bounds__(WTX * WTY) wave_stage_kernel(Dims d, Scalars sc, StageParams a) {
  const int i = blockIdx.x * WTX + threadIdx.x;
  const int j = blockIdx.y * WTY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  Loader<2> ld{a.src + c, nullptr, d.sy, d.sz, d.sv};
  double out[2];
  chemora_wave_point(ld, sc, out);
  stage_epilogue<2>(out, c, d.sv, a);
}

__global__ void __launch_bounds__(WTX * WTY) varc_stage_kernel(Dims d, Scalars sc, StageParams a) {
  const int i = blockIdx.x * WTX + threadIdx.x;
  const int j = blockIdx.y * WTY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  Loader<2> ld{a.src + c, a.coef + c, d.sy, d.sz, d.sv};
  double out[2];
  chemora_varc_point(ld, sc, out);
  stage_epilogue<2>(out, c, d.sv, a);
}

static dim3 wave_grid(const Dims& d) {
  return dim3((d.nx + WTX - 1) / WTX, (d.ny + WTY - 1) / WTY, d.nz);
}

int launch_wave_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  wave_stage_kernel<<<wave_grid(d), dim3(WTX, WTY), 0, s>>>(d, sc, a);
  return launched("wave_stage_kernel");
}

int launch_varc_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  varc_stage_kernel<<<wave_grid(d), dim3(WTX, WTY), 0, s>>>(d, sc, a);
  return launched("varc_stage_kernel");
}

}  // namespace chemora
