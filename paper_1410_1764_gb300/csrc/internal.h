// Internal declarations of libchemora (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "chemora.h"
#include "device_types.cuh"

namespace chemora {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);
#define CHEMORA_CUDA(call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return ::chemora::cuda_error(e_, #call); \
  } while (0)
// after a kernel launch: count it and check the launch status
int launched(const char* name, int n = 1);

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
enum HandleType : uint32_t {
  H_GRID = 0x47524944u,
  H_SYSTEM = 0x53595354u,
  H_BATCH = 0x42415443u,
  H_AMR = 0x414d5246u
};

struct chemora_grid_impl;
struct JitModule;  // run-time specialised stage kernels of one system

}  // namespace chemora

struct chemora_grid {
  uint32_t type;
  chemora::Dims d;
  int nvars;
  double dx;
  int64_t fsize;  // doubles per grid function
};

struct chemora_system {
  uint32_t type;
  chemora_grid* grid;
  int kind;
  int nvars;
  chemora_params params;
  chemora::Scalars sc;
  // RK4 scratch: acc, stage a, stage b (library-owned)
  double* scratch;
  // variable-speed coefficients (library-owned, 4 grid functions svar apart):
  // s = c^2 with ghosts, then G_d = D_d s on the interior
  double* coef;
  // device copy of a host state for chemora_rk4_step_host (library-owned)
  double* dev_state;
  // launch shape chosen by the autotuner (index into the kind's variants)
  int variant;
  // CUDA graph of one RK4 step (captured on cap_stream, replayed on the
  // caller's stream); key: state pointer, dt, variant
  cudaStream_t cap_stream;
  cudaGraph_t graph;
  cudaGraphExec_t graph_exec;
  double* graph_state;
  double graph_dt;
  int graph_variant;
  // run-time specialised stage kernels (NULL until chemora_system_specialize)
  chemora::JitModule* jit;
  int jit_on;
  // launch-chained RK4 steps of the order-4 scalar wave (wave_chain.cu):
  // its captured graphs, and whether chemora_rk4_step uses it
  void* chain;
  int chain_on;
  // profiling
  int profile_on;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used;
  double prof_ms;
  int64_t prof_launches;
};

namespace chemora {

Scalars make_scalars(double dx, const chemora_params& p);
int validate_system(int kind, int nvars, int nghost, int order);
int effective_order(int kind, const chemora_params& p);

// ghost fill of nvars grid functions (periodic image of the interior)
int fill_ghosts(const Dims& d, int nvars, double* state, cudaStream_t s);
int fill_ghosts_axes(const Dims& d, int nvars, double* state, int mask, cudaStream_t s);

int launch_stage(int kind, const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s,
                 int variant = 0);
int launch_wave_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant);
int launch_varc_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant);
// G_d = D_d s (4th-order centred) on the interior of 3 grid functions at G,
// svar apart; s with valid ghosts.
int launch_varc_grad(const Dims& d, double i12h, const double* s, double* G, cudaStream_t st);
int launch_bssn_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant);
int launch_wave_order_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s,
                            int variant);
int launch_wave1_stage(const Dims& d, const Scalars& sc, const StageParams& a, cudaStream_t s, int variant);

// A compiled launch shape of a stage kernel (tx x ty threads, min blocks/SM).
typedef int (*StageLaunchFn)(const Dims&, const Scalars&, const StageParams&, cudaStream_t);
struct LaunchVariant {
  int tx, ty, minb;
  StageLaunchFn launch;
  int xshare;  // 1: lanes share x-direction work (nx % tx == 0); 2: and y via
               // shared memory; 4: x lanes + z-march with a register queue of
               // z first differences (order-4 wave); 8: the one-point body on
               // a cp.async-staged tile with halos (order-4 wave; any nx)
};
extern const LaunchVariant kBssnVariants[];
extern const int kNumBssnVariants;
extern const LaunchVariant kWaveVariants[];
extern const int kNumWaveVariants;
extern const LaunchVariant kVarcVariants[];
extern const int kNumVarcVariants;
extern const LaunchVariant kWave1Variants[];
extern const int kNumWave1Variants;
int num_variants(int kind);
const LaunchVariant* variant_info(int kind, int v);

// Time the plausible launch shapes of kind's stage kernel on grid d (stage
// arguments p, written into p.acc / p.dst) and return the fastest in *best
// (left alone if none ran) and its time.  Synchronous.
int autotune_stage(int kind, const Dims& d, const Scalars& sc, const StageParams& p, cudaStream_t s, int* best,
                   float* best_ms);

// timing helpers for systems with profiling enabled
int prof_begin(chemora_system* sys, cudaStream_t s, cudaEvent_t* e0);
int prof_end(chemora_system* sys, cudaStream_t s, cudaEvent_t e0);

int ensure_scratch(chemora_system* sys);
void free_step_graph(chemora_system* sys);

// launch-chained RK4 steps of the order-4 scalar wave (wave_chain.cu)
bool chain_available(const chemora_system* sys);
int chain_rk4(chemora_system* sys, double* state, double dt, int nsteps, cudaStream_t s);
void chain_free(chemora_system* sys);

// run-time specialisation (jit.cu)
bool jit_active(const chemora_system* sys);
int jit_launch(chemora_system* sys, const StageParams& a, cudaStream_t s);
void jit_free(chemora_system* sys);

// Batched work-lists (patches.cu): a table of patches (grids inside one
// storage, each with its own extents and strides; the stage kernels compute
// the patch interior [g, n + g) per axis) and work items of up to 128
// consecutive interior points of one patch, x fastest.
struct PatchDesc {
  Dims d;
  int64_t offset;  // first double of the patch's state in the storage
  int64_t npts;    // interior points
};
struct WorkItem {
  int patch;
  int start;  // first interior point (linear, x fastest)
};
constexpr int kItemPoints = 128;
// Append the work items of patch q (npts interior points) to `items`.
void append_items(std::vector<WorkItem>& items, int q, int64_t npts);
// One persistent batched stage launch of a system of nvars variables (24:
// BSSN, 2: wave) over the device work-list `items` of the device patch table
// `pd`; `counter` (device, zero before the launch) hands out the items; bit
// 0 of *err is set for an item naming a patch outside the table, bit 1 when
// a block passed `limit` SM cycles (0: no limit).  src, yn, acc and dst of
// `p` are the storage bases; each patch's offset is added per item.
int launch_batch_stage(int nvars, const PatchDesc* pd, int npatch, const WorkItem* items, int nitems,
                       unsigned int* counter, int* err, long long limit, const Scalars& sc,
                       const StageParams& p, cudaStream_t s);

inline bool is_handle(const void* h, uint32_t t) {
  return h != nullptr && *reinterpret_cast<const uint32_t*>(h) == t;
}

}  // namespace chemora
