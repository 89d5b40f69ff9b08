// BSSN stage kernel: the generated Einstein-equation right-hand side (Sec. 3.4
// and Sec. 5 name the system; the body comes from gen/systems.py) fused with
// Kreiss-Oliger dissipation and the Runge-Kutta update.
//
// One thread per point.  The FP64 pipe is the bound on GB300 (two FP64 FMA
// per clock per SM), so a block of 128 threads with up to 255 registers each
// and two blocks per SM already keeps it busy; neighbour values come through
// the read-only data cache.
#include "stage.cuh"
#include "generated/gen_bssn.cuh"

namespace chemora {

constexpr int BTX = 32, BTY = 4;

__global__ void __launch_bounds__(BTX * BTY, 2) bssn_stage_kernel(Dims d, Scalars sc, StageParams a) {
  const int i = blockIdx.x * BTX + threadIdx.x;
  const int j = blockIdx.y * BTY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  Loader<24> ld{a.src + c, nullptr, d.sy, d.sz, d.sv};
  double out[24];
  chemora_bssn_point(ld, sc, out);
  stage_epilogue<24>(out, c, d.sv, a);
}

int launch_bssn_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s) {
  dim3 grid((d.nx + BTX - 1) / BTX, (d.ny + BTY - 1) / BTY, d.nz);
  bssn_stage_kernel<<<grid, dim3(BTX, BTY), 0, s>>>(d, sc, a);
  return launched("bssn_stage_kernel");
}

}  // namespace chemora
