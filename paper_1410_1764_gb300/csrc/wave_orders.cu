// Scalar-wave stage kernels of arbitrary finite-difference order (Sec.
// 3.2.2: "standard" operators of arbitrary order, the order fixed when the
// code is generated): the two-variable form at orders 2, 6, 8 (order 4 is in
// wave.cu) and the first-order form of Eq. 1 (u, rho, v_i) at orders 2, 4,
// 6, 8.  Bodies generated from gen/systems.py; every body is compiled in the
// same block shapes as the order-4 wave kernel so the autotuner can choose.
#include "internal.h"
#include "stage.cuh"
#include "generated/gen_wave_o2.cuh"
#include "generated/gen_wave_o6.cuh"
#include "generated/gen_wave_o8.cuh"
#include "generated/gen_wave1_o2.cuh"
#include "generated/gen_wave1_o4.cuh"
#include "generated/gen_wave1_o6.cuh"
#include "generated/gen_wave1_o8.cuh"

namespace chemora {

#define CHEMORA_BODY(NAME, NV, FN)                                                              \
  struct NAME {                                                                                 \
    static constexpr int nv = NV;                                                               \
    template <class LD, class OUT>                                                              \
    __device__ __forceinline__ static void eval(const LD& ld, const Scalars& sc, OUT& o) {      \
      FN(ld, sc, o);                                                                            \
    }                                                                                           \
  };

CHEMORA_BODY(WaveO2, 2, chemora_wave_o2_point)
CHEMORA_BODY(WaveO6, 2, chemora_wave_o6_point)
CHEMORA_BODY(WaveO8, 2, chemora_wave_o8_point)
CHEMORA_BODY(Wave1O2, 5, chemora_wave1_o2_point)
CHEMORA_BODY(Wave1O4, 5, chemora_wave1_o4_point)
CHEMORA_BODY(Wave1O6, 5, chemora_wave1_o6_point)
CHEMORA_BODY(Wave1O8, 5, chemora_wave1_o8_point)

template <class BODY, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) order_stage_kernel(Dims d, Scalars sc, StageParams a) {
  constexpr int NV = BODY::nv;
  const int i = blockIdx.x * TX + threadIdx.x;
  const int j = blockIdx.y * TY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  Loader<NV> ld{a.src + c, nullptr, d.sy, d.sz, d.sv};
  StageOutFma out = CHEMORA_STAGE_OUT_FMA(a, c, d.sv, sc);  // the wave systems' contracted update
  BODY::eval(ld, sc, out);
}

template <class BODY, int TX, int TY>
static int launch_order(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, d.nz);
  order_stage_kernel<BODY, TX, TY><<<grid, dim3(TX, TY), 0, s>>>(d, sc, a);
  return launched("order_stage_kernel");
}

#define CHEMORA_SHAPES(BODY)                                                                       \
  {{32, 8, 0, launch_order<BODY, 32, 8>},   {32, 4, 0, launch_order<BODY, 32, 4>},                 \
   {64, 4, 0, launch_order<BODY, 64, 4>},   {128, 2, 0, launch_order<BODY, 128, 2>},               \
   {32, 16, 0, launch_order<BODY, 32, 16>}, {16, 16, 0, launch_order<BODY, 16, 16>}}

constexpr int kOrderShapes = 6;
static const LaunchVariant kWaveO2[kOrderShapes] = CHEMORA_SHAPES(WaveO2);
static const LaunchVariant kWaveO6[kOrderShapes] = CHEMORA_SHAPES(WaveO6);
static const LaunchVariant kWaveO8[kOrderShapes] = CHEMORA_SHAPES(WaveO8);
static const LaunchVariant kWave1O2[kOrderShapes] = CHEMORA_SHAPES(Wave1O2);
static const LaunchVariant kWave1O6[kOrderShapes] = CHEMORA_SHAPES(Wave1O6);
static const LaunchVariant kWave1O8[kOrderShapes] = CHEMORA_SHAPES(Wave1O8);
const LaunchVariant kWave1Variants[kOrderShapes] = CHEMORA_SHAPES(Wave1O4);
const int kNumWave1Variants = kOrderShapes;

int launch_wave_order_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s,
                            int variant) {
  if (variant < 0 || variant >= kOrderShapes) variant = 0;
  switch (sc.order) {
    case 2: return kWaveO2[variant].launch(d, sc, a, s);
    case 6: return kWaveO6[variant].launch(d, sc, a, s);
    case 8: return kWaveO8[variant].launch(d, sc, a, s);
    default: return set_error(CHEMORA_EUNSUPPORTED, "scalar wave of order %d is not compiled", sc.order);
  }
}

int launch_wave1_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s,
                       int variant) {
  if (variant < 0 || variant >= kOrderShapes) variant = 0;
  switch (sc.order) {
    case 2: return kWave1O2[variant].launch(d, sc, a, s);
    case 4: return kWave1Variants[variant].launch(d, sc, a, s);
    case 6: return kWave1O6[variant].launch(d, sc, a, s);
    case 8: return kWave1O8[variant].launch(d, sc, a, s);
    default: return set_error(CHEMORA_EUNSUPPORTED, "first-order wave of order %d is not compiled", sc.order);
  }
}

}  // namespace chemora
