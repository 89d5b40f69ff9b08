// Autotuner for the stage kernels' launch shapes (the paper's GPU runtime
// does model-driven auto-tuning of the thread assignment, Sec. 3.2.3).
//
// Candidates are the compiled block shapes of the system's stage kernel.  A
// model ranks them by the threads they launch (x/y tile waste on ragged
// grids), by wave quantisation (blocks per SM slot count) and by the FP64
// instruction count of their body; candidates the model predicts more than
// 1.5x slower than its best are skipped, the rest are timed with CUDA
// events on the caller's grid (a middle RK stage, two repetitions after a
// warm-up) and the fastest is kept by the system.  Shapes of one body
// perform the same arithmetic; different bodies (direct, lane-, shared-
// memory- or z-queue-sharing) agree to rounding.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "generated/opcounts.inc"

namespace chemora {

// FP64 work of the xy-sharing prologue per point for blocks of ty rows: own
// y difference of 24 variables (1 sub each) and own z-derivative row of 11
// (2 subs + 1 fma: 3 instructions, 4 flops), plus the halo rows: 5 of the ty
// warp rows add 24 differences, 4 add 11 z rows.  Rounded to the nearest
// integer per point (ty = 8: 89 instructions, 105 flops).
static int64_t xy_prologue_instr(int ty) {
  return (int64_t)llround(24 + 33 + (5.0 * 24 + 4.0 * 33) / ty);
}
static int64_t xy_prologue_flops(int ty) {
  return (int64_t)llround(24 + 44 + (5.0 * 24 + 4.0 * 44) / ty);
}

static double model_cost(int kind, const Dims& d, const LaunchVariant& v, int sms) {
  // lane-sharing shapes need whole warps of x points
  if (v.xshare && v.xshare != 8 && d.nx % v.tx != 0) return 1e300;
  const double nbx = ceil((double)d.nx / v.tx), nby = ceil((double)d.ny / v.ty);
  const double blocks = nbx * nby * d.nz;
  const double threads = blocks * v.tx * v.ty;  // launched, including idle edge threads
  // resident blocks per SM: register-bound for BSSN (255 regs), thread-bound otherwise
  const int per_block = v.tx * v.ty;
  // resident blocks per SM: the register cap implied by minb for BSSN
  int bps = kind == CHEMORA_BSSN ? std::max(1, v.minb) : 2048 / per_block;
  if (bps < 1) bps = 1;
  const double waves = blocks / (double)(sms * bps);
  const double quant = waves < 1.0 ? 1.0 / std::max(waves, 1e-9) : ceil(waves) / waves;
  // x-sharing bodies issue about 11 % fewer FP64 instructions per point
  // (the x/z wave shapes: 24 of 30 FP64 instructions per point)
  const double work = v.xshare == 2 ? 0.81 : (v.xshare == 1 ? 0.89 : (v.xshare == 4 ? 0.8 : 1.0));
  return work * threads * (waves < 8.0 ? quant : 1.0 + 0.5 / waves);
}

int autotune_stage(int kind, const Dims& d, const Scalars& sc, const StageParams& p, cudaStream_t s, int* best,
                   float* best_ms) {
  int dev = 0, sms = 152;
  CHEMORA_CUDA(cudaGetDevice(&dev));
  CHEMORA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int nv = num_variants(kind);
  std::vector<double> cost(nv);
  double cmin = 1e300;
  for (int v = 0; v < nv; ++v) {
    cost[v] = model_cost(kind, d, *variant_info(kind, v), sms);
    cmin = std::min(cmin, cost[v]);
  }
  cudaEvent_t e0, e1;
  CHEMORA_CUDA(cudaEventCreate(&e0));
  CHEMORA_CUDA(cudaEventCreate(&e1));
  int rc = CHEMORA_OK;
  float best_t = 1e30f;
  for (int v = 0; v < nv && rc == CHEMORA_OK; ++v) {
    if (cost[v] > 1.5 * cmin) continue;
    if ((rc = launch_stage(kind, d, sc, p, s, v))) break;  // warm-up
    float tmin = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, s);
      if ((rc = launch_stage(kind, d, sc, p, s, v))) break;
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tmin = std::min(tmin, ms);
    }
    if (tmin < best_t) {
      best_t = tmin;
      *best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_ms) *best_ms = best_t;
  return rc;
}

}  // namespace chemora

using namespace chemora;

extern "C" {

int chemora_variant_count(int kind) { return num_variants(kind); }

int chemora_variant_info(int kind, int variant, int* tx, int* ty, int* min_blocks, int* sharing) {
  const LaunchVariant* v = variant_info(kind, variant);
  if (!v) return set_error(CHEMORA_EINVAL, "no launch shape %d for kind %d", variant, kind);
  if (tx) *tx = v->tx;
  if (ty) *ty = v->ty;
  if (min_blocks) *min_blocks = v->minb;
  if (sharing) *sharing = v->xshare;
  return CHEMORA_OK;
}

int chemora_system_opcount(chemora_system* sys, int64_t* fp64_instructions, int64_t* flops) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  const LaunchVariant* v = variant_info(sys->kind, sys->variant);
  if (sys->kind == CHEMORA_WAVE && sys->sc.order == 4 && v && v->xshare == 4 &&
      sys->grid->d.nx % v->tx == 0 && sys->grid->d.g >= 2) {
    // x-lane / z-queue body plus, per point, the queue's new difference and
    // its two combinations and the lane-halo difference
    if (fp64_instructions) *fp64_instructions = CHEMORA_OPS_WAVE_XZ_INSTR + 4;
    if (flops) *flops = CHEMORA_OPS_WAVE_XZ_FLOPS + 4;
    return CHEMORA_OK;
  }
  const bool xs = v && v->xshare && sys->grid->d.nx % v->tx == 0 && sys->grid->d.g >= 3;
  if (sys->kind == CHEMORA_BSSN && xs && v->xshare == 2) {
    // body plus the prologue's shared differences and z rows
    if (fp64_instructions) *fp64_instructions = CHEMORA_OPS_BSSN_XY_INSTR + xy_prologue_instr(v->ty);
    if (flops) *flops = CHEMORA_OPS_BSSN_XY_FLOPS + xy_prologue_flops(v->ty);
    return CHEMORA_OK;
  }
  if (sys->kind == CHEMORA_BSSN && xs) {
    if (fp64_instructions) *fp64_instructions = CHEMORA_OPS_BSSN_X_INSTR;
    if (flops) *flops = CHEMORA_OPS_BSSN_X_FLOPS;
    return CHEMORA_OK;
  }
  return chemora_opcount(sys->kind, fp64_instructions, flops);
}

int chemora_system_variant(chemora_system* sys, int set, int* variant, int* tx, int* ty) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (set >= 0) {
    if (set >= num_variants(sys->kind))
      return set_error(CHEMORA_EINVAL, "variant %d outside [0, %d)", set, num_variants(sys->kind));
    sys->variant = set;
  }
  const LaunchVariant* v = variant_info(sys->kind, sys->variant);
  if (variant) *variant = sys->variant;
  if (tx) *tx = v ? v->tx : 0;
  if (ty) *ty = v ? v->ty : 0;
  return CHEMORA_OK;
}

int chemora_autotune(chemora_system* sys, double* state, int* variant, double* best_ms, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (!state) return set_error(CHEMORA_EINVAL, "state is NULL");
  if (sys->kind == CHEMORA_WAVE_VARC && !sys->coef)
    return set_error(CHEMORA_EINVAL, "variable-speed system without a speed (chemora_system_set_speed)");
  int rc = ensure_scratch(sys);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Dims& d = sys->grid->d;
  if ((rc = fill_ghosts(d, sys->nvars, state, s))) return rc;
  // time a middle RK stage (mode 2: reads src, yn, acc; writes acc, dst),
  // the launch the RK4 driver repeats, into the RK scratch
  const size_t n = (size_t)sys->nvars * sys->grid->fsize;
  StageParams p{};
  p.src = state; p.yn = state; p.acc = sys->scratch; p.dst = sys->scratch + n;
  p.coef = sys->coef; p.c1 = 0.0; p.c2 = 0.0; p.mode = 2;
  int best = sys->variant;
  float best_t = 1e30f;
  rc = autotune_stage(sys->kind, d, sys->sc, p, s, &best, &best_t);
  cudaEvent_t e0, e1;
  CHEMORA_CUDA(cudaEventCreate(&e0));
  CHEMORA_CUDA(cudaEventCreate(&e1));
  if (rc == CHEMORA_OK) sys->variant = best;
  // The order-4 scalar wave may also run its RK4 steps as launch-chained
  // stage kernels: time 4 steps of a copy of the state both ways (graph
  // replay of the per-stage kernels and ghost fills; the chained stages) and
  // keep the faster.
  if (rc == CHEMORA_OK && chain_available(sys)) {
    const size_t bytes = n * sizeof(double);
    double* tmp = nullptr;
    if (cudaMalloc(&tmp, bytes) == cudaSuccess) {
      const double dt = 0.25 * sys->grid->dx;
      float tm[2] = {1e30f, 1e30f};
      for (int m = 0; m < 2 && rc == CHEMORA_OK; ++m) {
        sys->chain_on = m;
        for (int rep = 0; rep < 3 && rc == CHEMORA_OK; ++rep) {  // the first is a warm-up
          if (cudaMemcpyAsync(tmp, state, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            rc = cuda_error(cudaGetLastError(), "cudaMemcpyAsync");
            break;
          }
          cudaEventRecord(e0, s);
          if ((rc = chemora_rk4_step(sys, tmp, dt, 4, s))) break;
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) tm[m] = std::min(tm[m], ms);
        }
      }
      sys->chain_on = tm[1] < tm[0] ? 1 : 0;
      free_step_graph(sys);  // graphs captured for the copy
      chain_free(sys);
      cudaFree(tmp);
    } else {
      cudaGetLastError();
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (variant) *variant = best;
  if (best_ms) *best_ms = best_t;
  return CHEMORA_OK;
}

int chemora_system_set_chain(chemora_system* sys, int mode, int* active) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (mode < -1 || mode > 1) return set_error(CHEMORA_EINVAL, "mode must be -1 (query), 0 or 1");
  if (mode == 1 && !chain_available(sys))
    return set_error(CHEMORA_EUNSUPPORTED, "launch-chained RK4 steps exist for the order-4 scalar wave only");
  if (mode >= 0) sys->chain_on = mode;
  if (active) *active = sys->chain_on;
  return CHEMORA_OK;
}

}  // extern "C"
