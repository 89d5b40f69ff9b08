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
  StageOutFma out = CHEMORA_STAGE_OUT_FMA(a, c, d.sv, sc);
  chemora_wave_point(ld, sc, out);
}

// Loader of the variable-speed body: state variables 0-1, then the
// coefficient fields s, D_x s, D_y s, D_z s (svar apart) as variables 2-5.
struct VarcLoader {
  const double* __restrict__ p;  // centre point of variable 0
  const double* __restrict__ q;  // centre point of s
  int64_t sy, sz, sv;
  __device__ __forceinline__ double operator()(int v, int dx, int dy, int dz) const {
    const int64_t off = dx + dy * sy + dz * sz;
    if (v < 2) return __ldg(p + v * sv + off);
    return __ldg(q + (v - 2) * sv + off);
  }
};

template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) varc_stage_kernel(Dims d, Scalars sc, StageParams a) {
  const int i = blockIdx.x * TX + threadIdx.x;
  const int j = blockIdx.y * TY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  VarcLoader ld{a.src + c, a.coef + c, d.sy, d.sz, d.sv};
  StageOutFma out = CHEMORA_STAGE_OUT_FMA(a, c, d.sv, sc);
  chemora_varc_point(ld, sc, out);
}

// 2.5D blocking for the order-4 scalar wave: a warp is 32 consecutive x
// points of one row (x-direction first differences shared across lanes, as
// in the BSSN x-sharing body), and each thread marches ZB points along z
// keeping the z first differences e_m = u(z+m+1) - u(z+m), m = -2..1, of its
// own column in registers; the generated body (chemora_wave_xz_point) takes
// 12h^2 D_zz u = 15 (e_0 - e_-1) - (e_1 - e_-2).  Per point: one new z load
// and three FP64 operations for the queue instead of four loads and seven
// operations.  Requires nx % TX == 0 (every lane an interior point).
#include "generated/gen_wave_xz.cuh"

struct XZLoader : XLoader<2> {
  double qa[1], qb[1];  // e_0 - e_-1 and e_1 - e_-2 of u at the current z
};

template <int TX, int TY, int ZB>
__global__ void __launch_bounds__(TX * TY) wave_xz_kernel(Dims d, Scalars sc, StageParams a) {
  const int i = blockIdx.x * TX + threadIdx.x;
  const int j = blockIdx.y * TY + threadIdx.y;
  const int k0 = blockIdx.z * ZB;
  if (j >= d.ny) return;  // whole warps (a warp is one row)
  const double one = sc.k[CHEMORA_K_ONE];
  int64_t c = (int64_t)(k0 + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  const double* u = a.src + c;
  double e[4], ulast;
  {
    const double um2 = __ldg(u - 2 * d.sz), um1 = __ldg(u - d.sz), u0 = __ldg(u), u1 = __ldg(u + d.sz);
    ulast = __ldg(u + 2 * d.sz);
    e[0] = fma(um2, -one, um1);
    e[1] = fma(um1, -one, u0);
    e[2] = fma(u0, -one, u1);
    e[3] = fma(u1, -one, ulast);
  }
  const int lane = threadIdx.x & 31;
  // x halo of the lane-shared first differences: lanes 1, 2 hold x0-2, x0-1
  // and lane 3 holds x0+32 (lanes 0 and 4 repeat a neighbour: the radius-2
  // stencil needs no more, and with 2 ghost layers every read stays in the row)
  const int xo = lane == 0 ? -2 : (lane < 3 ? -3 : (lane == 3 ? 29 : (lane == 4 ? 28 : 0)));
#pragma unroll 1
  for (int kz = 0; kz < ZB; ++kz) {
    if (k0 + kz >= d.nz) break;  // uniform over the block
    XZLoader ld;
    ld.p = a.src + c;
    ld.sy = d.sy;
    ld.sz = d.sz;
    ld.sv = d.sv;
    ld.xo_dx = xo;
    ld.xo_d1 = 0;
    ld.qa[0] = fma(e[1], -one, e[2]);
    ld.qb[0] = fma(e[0], -one, e[3]);
    StageOutFma out = CHEMORA_STAGE_OUT_FMA(a, c, d.sv, sc);
    chemora_wave_xz_point(ld, sc, out);
    if (k0 + kz + 1 < d.nz) {  // advance the queue (u(z+3) is inside the ghost layers only then)
      const double unew = __ldg(a.src + c + 3 * d.sz);
      e[0] = e[1];
      e[1] = e[2];
      e[2] = e[3];
      e[3] = fma(ulast, -one, unew);
      ulast = unew;
    }
    c += d.sz;
  }
}

template <int TX, int TY, int ZB>
static int launch_wave_xz(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  if (d.nx % TX != 0 || d.g < 2)
    return set_error(CHEMORA_EUNSUPPORTED, "x/z-sharing wave kernel needs nx %% %d == 0", TX);
  dim3 grid(d.nx / TX, (d.ny + TY - 1) / TY, (d.nz + ZB - 1) / ZB);
  wave_xz_kernel<TX, TY, ZB><<<grid, dim3(TX, TY), 0, s>>>(d, sc, a);
  return launched("wave_xz_kernel");
}

// Staged tiles: the block's 32 x 8 tile of u with its 2-point halo, for the
// five planes k-2 .. k+2, is copied into shared memory with cp.async (the
// "xy tiles plus ghost halos" staging), then the one-point body reads every
// u neighbour from shared memory (rho, y_n and acc from global memory).
// Copies past a ragged grid edge are clamped to the last padded row and
// column (their values feed no live thread).
struct TileLoader {
  const double* tile;  // [5][TY + 4][TX + 4], this thread's point at [2][ty + 2][tx + 2]
  const double* rho;   // rho at this point
  int px, plane;       // tile row pitch and plane size in doubles
  __device__ __forceinline__ double operator()(int v, int dx, int dy, int dz) const {
    if (v == 0) return tile[dz * plane + dy * px + dx];
    return __ldg(rho + dx);  // the body reads rho at the point only (dx = dy = dz = 0)
  }
};

template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) wave_tile_kernel(Dims d, Scalars sc, StageParams a) {
  constexpr int PX = TX + 4, PY = TY + 4, PLANE = PX * PY;
  __shared__ __align__(16) double tile[5 * PLANE];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, k = blockIdx.z;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int xmax = d.nx + 2 * d.g - 1, ymax = d.ny + 2 * d.g - 1;  // last padded column / row
  for (int e = tid; e < 5 * PLANE; e += TX * TY) {
    const int pz = e / PLANE, r = e - pz * PLANE, py = r / PX, px = r - py * PX;
    const int gx = min(x0 - 2 + px + d.g, xmax), gy = min(y0 - 2 + py + d.g, ymax);
    const double* src = a.src + (int64_t)(k - 2 + pz + d.g) * d.sz + (int64_t)gy * d.sy + gx;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(tile + e);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int i = x0 + threadIdx.x, j = y0 + threadIdx.y;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  TileLoader ld{tile + 2 * PLANE + (threadIdx.y + 2) * PX + threadIdx.x + 2, a.src + d.sv + c, PX, PLANE};
  StageOutFma out = CHEMORA_STAGE_OUT_FMA(a, c, d.sv, sc);
  chemora_wave_point(ld, sc, out);
}

template <int TX, int TY>
static int launch_wave_tile(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, d.nz);
  wave_tile_kernel<TX, TY><<<grid, dim3(TX, TY), 0, s>>>(d, sc, a);
  return launched("wave_tile_kernel");
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
    {32, 8, 0, launch_wave_xz<32, 8, 8>, 4},   {32, 8, 0, launch_wave_xz<32, 8, 16>, 4},
    {32, 4, 0, launch_wave_xz<32, 4, 16>, 4},  {64, 4, 0, launch_wave_xz<64, 4, 32>, 4},
    {32, 16, 0, launch_wave_xz<32, 16, 8>, 4},
    {32, 8, 0, launch_wave_tile<32, 8>, 8},    {32, 4, 0, launch_wave_tile<32, 4>, 8},
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
  const LaunchVariant& v = kWaveVariants[variant];
  if (v.xshare == 4 && (d.nx % v.tx != 0 || d.g < 2)) return kWaveVariants[0].launch(d, sc, a, s);
  return v.launch(d, sc, a, s);
}

int launch_varc_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant) {
  if (variant < 0 || variant >= kNumVarcVariants) variant = 0;
  return kVarcVariants[variant].launch(d, sc, a, s);
}

}  // namespace chemora
