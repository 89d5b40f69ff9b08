// C ABI of libchemora: handles, validation, error reporting, the RK4 driver
// (Sec. 2: the time-integrator thorn, here fused into the stage kernels) with
// CUDA-graph replay, kernel timing, and the FP64 throughput probe.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "internal.h"
#include "generated/opcounts.inc"

namespace chemora {

static thread_local char g_err[512] = "";
static std::atomic<int64_t> g_launches{0};

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  return set_error(CHEMORA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int launched(const char* name, int n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, name);
  return CHEMORA_OK;
}

Scalars make_scalars(double dx, const chemora_params& p) {
  Scalars s;
  s.i12h = 1.0 / (12.0 * dx);
  s.i12h2 = 1.0 / (12.0 * dx * dx);
  s.i144h2 = 1.0 / (144.0 * dx * dx);
  s.ko_scale = p.eps_diss / (64.0 * dx);
  s.eta = p.eta;
  s.slicing = p.slicing;
  s.shift = p.shift;
  s.ih = 1.0 / dx;
  s.ih2 = 1.0 / (dx * dx);
  s.order = p.fd_order ? p.fd_order : 4;
  for (int i = 0; i < CHEMORA_NK; ++i) s.k[i] = kChemoraK[i];
  return s;
}

static int nvars_of(int kind) {
  switch (kind) {
    case CHEMORA_WAVE:
    case CHEMORA_WAVE_VARC: return 2;
    case CHEMORA_BSSN: return 24;
    case CHEMORA_WAVE1: return 5;
    default: return -1;
  }
}

int effective_order(int kind, const chemora_params& p) {
  (void)kind;
  return p.fd_order ? p.fd_order : 4;
}

static int ghosts_of(int kind, int order) {
  if (kind == CHEMORA_BSSN) return 3;
  if (kind == CHEMORA_WAVE_VARC) return 2;
  return order / 2;
}

int validate_system(int kind, int nvars, int nghost, int order) {
  const int nv = nvars_of(kind);
  if (nv < 0) return set_error(CHEMORA_EINVAL, "unknown system kind %d", kind);
  if (nvars != nv)
    return set_error(CHEMORA_EINVAL, "system kind %d needs nvars=%d, grid has %d", kind, nv, nvars);
  const bool any_order = kind == CHEMORA_WAVE || kind == CHEMORA_WAVE1;
  if (any_order ? (order != 2 && order != 4 && order != 6 && order != 8) : order != 4)
    return set_error(CHEMORA_EINVAL, "system kind %d does not support finite-difference order %d", kind,
                     order);
  if (nghost < ghosts_of(kind, order))
    return set_error(CHEMORA_EINVAL, "system kind %d needs nghost>=%d, grid has %d", kind,
                     ghosts_of(kind, order), nghost);
  return CHEMORA_OK;
}

int launch_stage(int kind, const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s,
                 int variant) {
  switch (kind) {
    case CHEMORA_WAVE: return launch_wave_stage(d, sc, a, s, variant);
    case CHEMORA_WAVE_VARC: return launch_varc_stage(d, sc, a, s, variant);
    case CHEMORA_BSSN: return launch_bssn_stage(d, sc, a, s, variant);
    case CHEMORA_WAVE1: return launch_wave1_stage(d, sc, a, s, variant);
    default: return set_error(CHEMORA_EINVAL, "unknown system kind %d", kind);
  }
}

int num_variants(int kind) {
  switch (kind) {
    case CHEMORA_WAVE: return kNumWaveVariants;
    case CHEMORA_WAVE_VARC: return kNumVarcVariants;
    case CHEMORA_BSSN: return kNumBssnVariants;
    case CHEMORA_WAVE1: return kNumWave1Variants;
    default: return 0;
  }
}

const LaunchVariant* variant_info(int kind, int v) {
  if (v < 0 || v >= num_variants(kind)) return nullptr;
  switch (kind) {
    case CHEMORA_WAVE: return &kWaveVariants[v];
    case CHEMORA_WAVE_VARC: return &kVarcVariants[v];
    case CHEMORA_WAVE1: return &kWave1Variants[v];
    default: return &kBssnVariants[v];
  }
}

int ensure_scratch(chemora_system* sys) {
  if (sys->scratch) return CHEMORA_OK;
  const size_t n = (size_t)sys->nvars * sys->grid->fsize;
  cudaError_t e = cudaMalloc(&sys->scratch, 3 * n * sizeof(double));
  if (e != cudaSuccess) {
    sys->scratch = nullptr;
    cudaGetLastError();
    return set_error(CHEMORA_ENOMEM, "RK4 scratch of %zu bytes: %s", 3 * n * sizeof(double),
                     cudaGetErrorString(e));
  }
  // zero once so that never-written ghost cells hold defined values
  CHEMORA_CUDA(cudaMemset(sys->scratch, 0, 3 * n * sizeof(double)));
  return CHEMORA_OK;
}

static int next_event(chemora_system* sys, cudaEvent_t* ev) {
  if (sys->ev_used < sys->ev_pool.size()) {
    *ev = sys->ev_pool[sys->ev_used++];
    return CHEMORA_OK;
  }
  cudaEvent_t e;
  CHEMORA_CUDA(cudaEventCreate(&e));
  sys->ev_pool.push_back(e);
  sys->ev_used++;
  *ev = e;
  return CHEMORA_OK;
}

int prof_begin(chemora_system* sys, cudaStream_t s, cudaEvent_t* e0) {
  *e0 = nullptr;
  if (!sys->profile_on) return CHEMORA_OK;
  int rc = next_event(sys, e0);
  if (rc) return rc;
  CHEMORA_CUDA(cudaEventRecord(*e0, s));
  return CHEMORA_OK;
}

int prof_end(chemora_system* sys, cudaStream_t s, cudaEvent_t e0) {
  if (!sys->profile_on || !e0) return CHEMORA_OK;
  cudaEvent_t e1;
  int rc = next_event(sys, &e1);
  if (rc) return rc;
  CHEMORA_CUDA(cudaEventRecord(e1, s));
  return CHEMORA_OK;
}

static int run_stage(chemora_system* sys, const StageParams& a, cudaStream_t s) {
  cudaEvent_t e0;
  int rc = prof_begin(sys, s, &e0);
  if (rc) return rc;
  rc = jit_active(sys) ? jit_launch(sys, a, s)
                       : launch_stage(sys->kind, sys->grid->d, sys->sc, a, s, sys->variant);
  if (rc) return rc;
  return prof_end(sys, s, e0);
}

// One RK4 step: four fused stages, each preceded by a ghost fill of the
// buffer its stencils read.  Buffers: Y (caller's state), A (accumulator),
// Sa/Sb (stage states, alternating so no stage reads what it writes).
static int rk4_one(chemora_system* sys, double* Y, double dt, cudaStream_t s) {
  const Dims& d = sys->grid->d;
  const int nv = sys->nvars;
  const size_t n = (size_t)nv * sys->grid->fsize;
  double* A = sys->scratch;
  double* Sa = sys->scratch + n;
  double* Sb = sys->scratch + 2 * n;
  int rc;
  StageParams p{};
  p.coef = sys->coef;
  if ((rc = fill_ghosts(d, nv, Y, s))) return rc;
  p.src = Y; p.yn = Y; p.acc = A; p.dst = Sa; p.c1 = 0.0; p.c2 = 0.5 * dt; p.mode = 1;
  if ((rc = run_stage(sys, p, s))) return rc;
  if ((rc = fill_ghosts(d, nv, Sa, s))) return rc;
  p.src = Sa; p.dst = Sb; p.c2 = 0.5 * dt; p.mode = 2;
  if ((rc = run_stage(sys, p, s))) return rc;
  if ((rc = fill_ghosts(d, nv, Sb, s))) return rc;
  p.src = Sb; p.dst = Sa; p.c2 = dt; p.mode = 3;
  if ((rc = run_stage(sys, p, s))) return rc;
  if ((rc = fill_ghosts(d, nv, Sa, s))) return rc;
  p.src = Sa; p.dst = Y; p.c1 = dt / 6.0; p.c2 = 0.0; p.mode = 4;
  return run_stage(sys, p, s);
}

void free_step_graph(chemora_system* sys) {
  if (sys->graph_exec) cudaGraphExecDestroy(sys->graph_exec);
  if (sys->graph) cudaGraphDestroy(sys->graph);
  sys->graph_exec = nullptr;
  sys->graph = nullptr;
  sys->graph_state = nullptr;
}

// One RK4 step captured into a CUDA graph (on a private stream: the legacy
// default stream cannot be captured), cached per (state, dt, variant).
static int step_graph(chemora_system* sys, double* state, double dt) {
  if (sys->graph_exec && sys->graph_state == state && sys->graph_dt == dt &&
      sys->graph_variant == sys->variant)
    return CHEMORA_OK;
  free_step_graph(sys);
  if (!sys->cap_stream) CHEMORA_CUDA(cudaStreamCreateWithFlags(&sys->cap_stream, cudaStreamNonBlocking));
  CHEMORA_CUDA(cudaStreamBeginCapture(sys->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = rk4_one(sys, state, dt, sys->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(sys->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  sys->graph = g;
  CHEMORA_CUDA(cudaGraphInstantiate(&sys->graph_exec, g, 0));
  sys->graph_state = state;
  sys->graph_dt = dt;
  sys->graph_variant = sys->variant;
  return CHEMORA_OK;
}

}  // namespace chemora

using namespace chemora;

extern "C" {

int chemora_grid_create(int nx, int ny, int nz, int nvars, int nghost, double dx,
                        chemora_grid** out) {
  if (!out) return set_error(CHEMORA_EINVAL, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || nvars < 1 || nghost < 1)
    return set_error(CHEMORA_EINVAL, "grid sizes must be >= 1 (nx=%d ny=%d nz=%d nvars=%d nghost=%d)",
                     nx, ny, nz, nvars, nghost);
  if (!(dx > 0.0) || !isfinite(dx)) return set_error(CHEMORA_EINVAL, "dx must be finite and > 0");
  if (nx > 65535 * 32 || ny > 65535 * 4 || nz > 65535)
    return set_error(CHEMORA_EINVAL, "grid extent beyond the launch limits");
  const int64_t px = (int64_t)nx + 2 * nghost, py = (int64_t)ny + 2 * nghost,
                pz = (int64_t)nz + 2 * nghost;
  const int64_t fsize = px * py * pz;
  if (fsize * nvars > ((int64_t)1 << 40)) return set_error(CHEMORA_EINVAL, "state too large");
  chemora_grid* g = new (std::nothrow) chemora_grid();
  if (!g) return set_error(CHEMORA_ENOMEM, "host allocation");
  g->type = H_GRID;
  g->d.nx = nx; g->d.ny = ny; g->d.nz = nz; g->d.g = nghost;
  g->d.sy = px; g->d.sz = px * py; g->d.sv = fsize;
  g->nvars = nvars;
  g->dx = dx;
  g->fsize = fsize;
  *out = g;
  return CHEMORA_OK;
}

int chemora_grid_layout(const chemora_grid* grid, int64_t* sy, int64_t* sz, int64_t* svar) {
  if (!is_handle(grid, H_GRID)) return set_error(CHEMORA_EINVAL, "not a grid handle");
  if (sy) *sy = grid->d.sy;
  if (sz) *sz = grid->d.sz;
  if (svar) *svar = grid->d.sv;
  return CHEMORA_OK;
}

int chemora_system_create(chemora_grid* grid, int kind, const chemora_params* params,
                          chemora_system** out) {
  if (!out) return set_error(CHEMORA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!is_handle(grid, H_GRID)) return set_error(CHEMORA_EINVAL, "not a grid handle");
  chemora_params p = {0.1, 2.0, 0, 0, 0};
  if (params) p = *params;
  int rc = validate_system(kind, grid->nvars, grid->d.g, effective_order(kind, p));
  if (rc) return rc;
  if (p.slicing < 0 || p.slicing > 2 || p.shift < 0 || p.shift > 1 || !isfinite(p.eps_diss) ||
      !isfinite(p.eta))
    return set_error(CHEMORA_EINVAL, "bad params (slicing %d, shift %d)", p.slicing, p.shift);
  chemora_system* s = new (std::nothrow) chemora_system();
  if (!s) return set_error(CHEMORA_ENOMEM, "host allocation");
  s->type = H_SYSTEM;
  s->grid = grid;
  s->kind = kind;
  s->nvars = grid->nvars;
  s->params = p;
  s->sc = make_scalars(grid->dx, p);
  *out = s;
  return CHEMORA_OK;
}

int chemora_fill_ghosts(chemora_system* sys, double* state, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (!state) return set_error(CHEMORA_EINVAL, "state is NULL");
  return fill_ghosts(sys->grid->d, sys->nvars, state, (cudaStream_t)stream);
}

int chemora_rhs(chemora_system* sys, const double* state, double* rhs, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (!state || !rhs) return set_error(CHEMORA_EINVAL, "NULL state or rhs");
  if (state == rhs) return set_error(CHEMORA_EINVAL, "state and rhs must not overlap");
  if (sys->kind == CHEMORA_WAVE_VARC && !sys->coef)
    return set_error(CHEMORA_EINVAL, "variable-speed system without a speed (chemora_system_set_speed)");
  StageParams p{};
  p.src = state; p.dst = rhs; p.coef = sys->coef; p.mode = 0;
  return run_stage(sys, p, (cudaStream_t)stream);
}

int chemora_rk4_step(chemora_system* sys, double* state, double dt, int nsteps, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (!state) return set_error(CHEMORA_EINVAL, "state is NULL");
  if (nsteps < 0) return set_error(CHEMORA_EINVAL, "nsteps < 0");
  if (!isfinite(dt)) return set_error(CHEMORA_EINVAL, "dt not finite");
  if (sys->kind == CHEMORA_WAVE_VARC && !sys->coef)
    return set_error(CHEMORA_EINVAL, "variable-speed system without a speed (chemora_system_set_speed)");
  int rc = ensure_scratch(sys);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  CHEMORA_CUDA(cudaStreamIsCapturing(s, &cst));
  // The scalar wave's launch-chained path (small grids, chosen by the autotuner).
  if (sys->chain_on && chain_available(sys) && !sys->profile_on && cst == cudaStreamCaptureStatusNone)
    return chain_rk4(sys, state, dt, nsteps, s);
  // Plain launches while profiling (events bracket each stage) or when the
  // caller is capturing the stream itself; otherwise replay a captured step.
  if (sys->profile_on || cst != cudaStreamCaptureStatusNone || nsteps < 2) {
    for (int n = 0; n < nsteps; ++n)
      if ((rc = rk4_one(sys, state, dt, s))) return rc;
    return fill_ghosts(sys->grid->d, sys->nvars, state, s);
  }
  if ((rc = step_graph(sys, state, dt))) return rc;
  for (int n = 0; n < nsteps; ++n) {
    CHEMORA_CUDA(cudaGraphLaunch(sys->graph_exec, s));
    if ((rc = launched("cudaGraphLaunch(RK4 step)", 8))) return rc;
  }
  return fill_ghosts(sys->grid->d, sys->nvars, state, s);
}

int chemora_rk4_step_host(chemora_system* sys, double* host_state, double dt, int nsteps,
                          void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (!host_state) return set_error(CHEMORA_EINVAL, "host_state is NULL");
  const size_t bytes = (size_t)sys->nvars * sys->grid->fsize * sizeof(double);
  if (!sys->dev_state) {
    cudaError_t e = cudaMalloc(&sys->dev_state, bytes);
    if (e != cudaSuccess) {
      sys->dev_state = nullptr;
      cudaGetLastError();
      return set_error(CHEMORA_ENOMEM, "device state of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  CHEMORA_CUDA(cudaMemcpyAsync(sys->dev_state, host_state, bytes, cudaMemcpyHostToDevice, s));
  int rc = chemora_rk4_step(sys, sys->dev_state, dt, nsteps, stream);
  if (rc) return rc;
  CHEMORA_CUDA(cudaMemcpyAsync(host_state, sys->dev_state, bytes, cudaMemcpyDeviceToHost, s));
  CHEMORA_CUDA(cudaStreamSynchronize(s));
  return CHEMORA_OK;
}

int chemora_fill_ghosts_axes(chemora_system* sys, double* state, int axes, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (!state) return set_error(CHEMORA_EINVAL, "state is NULL");
  if (axes < 0 || axes > 7) return set_error(CHEMORA_EINVAL, "axes must be a mask of bits 0-2");
  if (axes == 0) return CHEMORA_OK;
  return fill_ghosts_axes(sys->grid->d, sys->nvars, state, axes, (cudaStream_t)stream);
}

int chemora_stage(chemora_system* sys, int mode, const double* src, const double* yn, double* acc,
                  double* dst, double c1, double c2, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (mode < 0 || mode > 4) return set_error(CHEMORA_EINVAL, "mode must be 0..4");
  if (!src || !dst || (mode > 0 && (!yn || !acc)))
    return set_error(CHEMORA_EINVAL, "NULL buffer for stage mode %d", mode);
  if (src == dst) return set_error(CHEMORA_EINVAL, "src and dst must not overlap");
  if (!isfinite(c1) || !isfinite(c2)) return set_error(CHEMORA_EINVAL, "non-finite coefficient");
  if (sys->kind == CHEMORA_WAVE_VARC && !sys->coef)
    return set_error(CHEMORA_EINVAL, "variable-speed system without a speed (chemora_system_set_speed)");
  StageParams p{};
  p.src = src; p.yn = yn; p.acc = acc; p.dst = dst; p.coef = sys->coef;
  p.c1 = c1; p.c2 = c2; p.mode = mode;
  return run_stage(sys, p, (cudaStream_t)stream);
}

int chemora_profile_enable(chemora_system* sys, int on) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  sys->profile_on = on ? 1 : 0;
  return CHEMORA_OK;
}

int chemora_profile_read(chemora_system* sys, double* total_ms, int64_t* launches, int reset) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  for (size_t q = 0; q + 1 < sys->ev_used; q += 2) {
    CHEMORA_CUDA(cudaEventSynchronize(sys->ev_pool[q + 1]));
    float ms = 0.f;
    CHEMORA_CUDA(cudaEventElapsedTime(&ms, sys->ev_pool[q], sys->ev_pool[q + 1]));
    sys->prof_ms += ms;
    sys->prof_launches += 1;
  }
  sys->ev_used = 0;
  if (total_ms) *total_ms = sys->prof_ms;
  if (launches) *launches = sys->prof_launches;
  if (reset) {
    sys->prof_ms = 0.0;
    sys->prof_launches = 0;
  }
  return CHEMORA_OK;
}

int64_t chemora_launch_count(void) { return g_launches.load(); }

int chemora_opcount(int kind, int64_t* fp64_instructions, int64_t* flops) {
  int64_t i = -1, f = -1;
  switch (kind) {
    case CHEMORA_WAVE: i = CHEMORA_OPS_WAVE_INSTR; f = CHEMORA_OPS_WAVE_FLOPS; break;
    case CHEMORA_WAVE_VARC: i = CHEMORA_OPS_VARC_INSTR; f = CHEMORA_OPS_VARC_FLOPS; break;
    case CHEMORA_BSSN: i = CHEMORA_OPS_BSSN_INSTR; f = CHEMORA_OPS_BSSN_FLOPS; break;
    case CHEMORA_WAVE1: i = CHEMORA_OPS_WAVE1_INSTR; f = CHEMORA_OPS_WAVE1_FLOPS; break;
    default: return set_error(CHEMORA_EINVAL, "unknown system kind %d", kind);
  }
  if (fp64_instructions) *fp64_instructions = i;
  if (flops) *flops = f;
  return CHEMORA_OK;
}

const char* chemora_last_error(void) { return g_err; }

}  // extern "C"
