// Plain device-side types shared by the ahead-of-time kernels and the
// run-time specialised ones: grid dimensions and strides, the scalars the
// generated point bodies read, and the arguments of a fused stage.  No host
// headers, so the run-time compiler (NVRTC) can include this file too.
#pragma once

#if defined(__CUDACC_RTC__)
typedef long long int64_t;
#else
#include <stdint.h>
#endif

#include "generated/gen_constants.cuh"  // CHEMORA_NK, CHEMORA_K_*

namespace chemora {

struct Dims {
  int nx, ny, nz, g;
  int64_t sy, sz, sv;  // strides in doubles
};

// Runtime scalars read by the generated point bodies (names match the
// generator's symbols).
struct Scalars {
  double i12h, i12h2, i144h2, ko_scale, eta;
  int slicing, shift;
  double ih, ih2;  // 1/h, 1/h^2 (arbitrary-order stencils)
  int order;       // finite-difference order of the wave systems
  // numeric constants of the generated bodies (gen_constants.cuh): every
  // FP64 add, subtract and multiply is issued as an fma with an operand
  // from this table, which the compiler cannot fold into an immediate
  double k[CHEMORA_NK];
};

// The constant table alone, as a kernel parameter of the run-time
// specialised kernels (whose other scalars are compile-time constants).
struct KTable {
  double k[CHEMORA_NK];
};

// One fused stage kernel over the interior (k = RHS(src)):
//   mode 0: dst = k
//   mode 1: acc = k;        dst = yn + c2 k        (c2 = dt/2)
//   mode 2: acc += 2k;      dst = yn + c2 k        (c2 = dt/2)
//   mode 3: acc += 2k;      dst = yn + c2 k        (c2 = dt)
//   mode 4: dst = yn + c1 (acc + k)                (c1 = dt/6)
struct StageParams {
  const double* src;
  const double* yn;
  double* acc;
  double* dst;
  const double* coef;  // coefficient grid functions (variable-speed wave: s, D_x s, D_y s, D_z s), else NULL
  double c1, c2;
  int mode;
};

// Bytes of dynamic shared memory of the BSSN x/y-sharing stage body for
// blocks of tx x ty threads: the y first differences [24][ty + 5][tx] and
// the z-derivative rows [11][ty + 4][tx].
__host__ __device__ constexpr unsigned bssn_xy_smem_bytes(int tx, int ty) {
  return (unsigned)((24 * (ty + 5) + 11 * (ty + 4)) * tx * sizeof(double));
}

}  // namespace chemora
