// Batched patches: many independent periodic grids of uneven sizes (the
// patches of an AMR or multi-block driver, Sec. 4) advanced together.
//
// mode 0 (batched): per RK stage one ghost-fill launch over every patch and
// one persistent stage launch.  The persistent kernel's blocks pull work
// items -- 128 consecutive interior points of one patch, x fastest -- from a
// work-list with an atomic counter, so uneven patches keep every SM busy and
// no thread idles on a partial x-tile.  The loop is bounded by the item count (the
// counter only grows), and an item naming a patch outside the table sets a
// device error word instead of touching memory.  The whole RK4 step is
// captured once in a CUDA graph and replayed.
// mode 1 (per patch): the single-grid kernels launched patch by patch, stage
// by stage (the schedule a driver without batching would use).
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "internal.h"
#include "stage.cuh"
#include "generated/gen_bssn.cuh"
#include "generated/gen_wave.cuh"

struct chemora_batch {
  uint32_t type;
  int kind, nvars, npatch, nghost;
  double dx;
  chemora::Scalars sc;
  std::vector<chemora::PatchDesc> host_pd;
  int64_t total;  // doubles per batch state
  double* state;  // library-owned batch storage
  double* scratch;  // acc, stage a, stage b
  chemora::PatchDesc* dev_pd;
  chemora::WorkItem* items;
  int nitems;
  unsigned int* counters;  // one per stage of a step
  int* err;                // device error word: bit 0 bad work item, bit 1 time limit
  long long limit_cycles;  // time limit of a persistent stage launch in SM cycles (0: none)
  cudaStream_t cap_stream;  // private stream the step graph is captured on
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  double graph_dt;
  int graph_kernels;
};

namespace chemora {

// one block of 128 threads (kItemPoints) per work item

template <int NV>
struct BatchBody;

template <>
struct BatchBody<24> {
  template <class LD, class OUT>
  __device__ __forceinline__ static void eval(const LD& ld, const Scalars& sc, OUT& out) {
    chemora_bssn_point(ld, sc, out);
  }
};

template <>
struct BatchBody<2> {
  template <class LD, class OUT>
  __device__ __forceinline__ static void eval(const LD& ld, const Scalars& sc, OUT& out) {
    chemora_wave_point(ld, sc, out);
  }
};

// MODE: the RK stage mode compiled in (its update's branches fold), or -1
// for the mode of the stage arguments.
template <int NV, int MODE>
__global__ void __launch_bounds__(128, 3)
batch_stage_kernel(const PatchDesc* __restrict__ pd, int npatch, const WorkItem* __restrict__ items,
                   int nitems, unsigned int* counter, int* err, long long limit, Scalars sc,
                   StageParams base_in) {
  StageParams base = base_in;
  if (MODE >= 0) base.mode = MODE;
  __shared__ unsigned int s_item;
  const long long t0 = clock64();
  for (int iter = 0; iter <= nitems; ++iter) {  // bounded: one counter value per pass
    if (threadIdx.x == 0) {
      // past the time limit the block takes no more items and reports it
      if (limit > 0 && clock64() - t0 > limit) {
        atomicOr(err, 2);
        s_item = (unsigned)nitems;
      } else {
        s_item = atomicAdd(counter, 1u);
      }
    }
    __syncthreads();
    const unsigned int it = s_item;
    __syncthreads();
    if (it >= (unsigned)nitems) break;
    const WorkItem w = items[it];
    if (w.patch < 0 || w.patch >= npatch) {
      if (threadIdx.x == 0) atomicOr(err, 1);
      continue;
    }
    const PatchDesc P = pd[w.patch];
    const int64_t lin = (int64_t)w.start + threadIdx.x;
    if (w.start < 0 || lin >= P.npts) continue;
    const int64_t plane = (int64_t)P.d.nx * P.d.ny;
    const int k = (int)(lin / plane);
    const int64_t r = lin - (int64_t)k * plane;
    const int j = (int)(r / P.d.nx);
    const int i = (int)(r - (int64_t)j * P.d.nx);
    const int64_t c = P.offset + (int64_t)(k + P.d.g) * P.d.sz + (int64_t)(j + P.d.g) * P.d.sy + (i + P.d.g);
    Loader<NV> ld{base.src + c, nullptr, P.d.sy, P.d.sz, P.d.sv};
    if (NV == 2) {  // the scalar wave's update (StageOutFma), as in its single-grid kernels
      StageOutFma out = CHEMORA_STAGE_OUT_FMA(base, c, P.d.sv, sc);
      BatchBody<NV>::eval(ld, sc, out);
    } else {
      StageOut out = CHEMORA_STAGE_OUT(base, c, P.d.sv, sc);
      BatchBody<NV>::eval(ld, sc, out);
    }
  }
}

__device__ __forceinline__ int bwrap(int i, int n, int g) {
  int r = (i - g) % n;
  return (r < 0 ? r + n : r) + g;
}

// Ghost fill of every patch and variable: blockIdx.y = patch, blockIdx.z = variable.
__global__ void batch_ghost_kernel(double* __restrict__ base, const PatchDesc* __restrict__ pd) {
  const PatchDesc P = pd[blockIdx.y];
  const Dims d = P.d;
  double* f = base + P.offset + (int64_t)blockIdx.z * d.sv;
  const int g = d.g;
  const int64_t px = d.nx + 2 * g, py = d.ny + 2 * g;
  const int64_t zslab = 2 * g * py * px;
  const int64_t yslab = (int64_t)d.nz * 2 * g * px;
  const int64_t total = zslab + yslab + (int64_t)d.nz * d.ny * 2 * g;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    if (t < zslab) {
      int64_t kk = t / (py * px), rem = t - kk * py * px;
      k = (int)(kk < g ? kk : kk + d.nz);
      j = (int)(rem / px);
      i = (int)(rem - (int64_t)j * px);
    } else if (t < zslab + yslab) {
      int64_t u = t - zslab;
      int64_t kk = u / (2 * g * px), rem = u - kk * 2 * g * px;
      k = (int)kk + g;
      int jj = (int)(rem / px);
      j = jj < g ? jj : jj + d.ny;
      i = (int)(rem - (int64_t)jj * px);
    } else {
      int64_t u = t - zslab - yslab;
      int64_t kk = u / ((int64_t)d.ny * 2 * g), rem = u - kk * d.ny * 2 * g;
      k = (int)kk + g;
      j = (int)(rem / (2 * g)) + g;
      int ii = (int)(rem % (2 * g));
      i = ii < g ? ii : ii + d.nx;
    }
    f[(int64_t)k * d.sz + (int64_t)j * d.sy + i] =
        f[(int64_t)bwrap(k, d.nz, g) * d.sz + (int64_t)bwrap(j, d.ny, g) * d.sy + bwrap(i, d.nx, g)];
  }
}

static int batch_ghosts(chemora_batch* b, double* base, cudaStream_t s) {
  dim3 grid(8, b->npatch, b->nvars);
  batch_ghost_kernel<<<grid, 256, 0, s>>>(base, b->dev_pd);
  return launched("batch_ghost_kernel");
}

static int persistent_blocks() {
  static int cached = 0;
  if (cached) return cached;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    sms = 152;
  cached = 3 * sms;  // three 128-thread blocks per SM (168 registers; measured best of 2-4)
  return cached;
}

struct BatchLaunch {
  const PatchDesc* pd;
  int npatch;
  const WorkItem* items;
  int nitems;
  unsigned int* counter;
  int* err;
  long long limit;
};

template <int NV, int MODE>
static void launch_batch_mode(const BatchLaunch& L, const Scalars& sc, const StageParams& p, cudaStream_t s) {
  batch_stage_kernel<NV, MODE><<<persistent_blocks(), kItemPoints, 0, s>>>(L.pd, L.npatch, L.items, L.nitems,
                                                                          L.counter, L.err, L.limit, sc, p);
}

template <int NV>
static void launch_batch_nv(const BatchLaunch& L, const Scalars& sc, const StageParams& p, cudaStream_t s) {
  switch (p.mode) {
    case 1: launch_batch_mode<NV, 1>(L, sc, p, s); break;
    case 2: launch_batch_mode<NV, 2>(L, sc, p, s); break;
    case 3: launch_batch_mode<NV, 3>(L, sc, p, s); break;
    case 4: launch_batch_mode<NV, 4>(L, sc, p, s); break;
    default: launch_batch_mode<NV, -1>(L, sc, p, s); break;
  }
}

int launch_batch_stage(int nvars, const PatchDesc* pd, int npatch, const WorkItem* items, int nitems,
                       unsigned int* counter, int* err, long long limit, const Scalars& sc,
                       const StageParams& p, cudaStream_t s) {
  const BatchLaunch L{pd, npatch, items, nitems, counter, err, limit};
  if (nvars == 24)
    launch_batch_nv<24>(L, sc, p, s);
  else if (nvars == 2)
    launch_batch_nv<2>(L, sc, p, s);
  else
    return set_error(CHEMORA_EINVAL, "batched stage kernels exist for 24 (BSSN) and 2 (wave) variables");
  return launched("batch_stage_kernel");
}

void append_items(std::vector<WorkItem>& items, int q, int64_t npts) {
  for (int64_t st = 0; st < npts; st += kItemPoints) items.push_back(WorkItem{q, (int)st});
}

static int batch_stage(chemora_batch* b, const StageParams& p, int stage, cudaStream_t s) {
  return launch_batch_stage(b->nvars, b->dev_pd, b->npatch, b->items, b->nitems, b->counters + stage, b->err,
                            b->limit_cycles, b->sc, p, s);
}

// One RK4 step of every patch, batched: 4 x (ghost fill + persistent stage).
static int batch_rk4_one(chemora_batch* b, double dt, cudaStream_t s) {
  const int64_t n = b->total;
  double* Y = b->state;
  double* A = b->scratch;
  double* Sa = b->scratch + n;
  double* Sb = b->scratch + 2 * n;
  int rc;
  CHEMORA_CUDA(cudaMemsetAsync(b->counters, 0, 4 * sizeof(unsigned int), s));
  StageParams p{};
  if ((rc = batch_ghosts(b, Y, s))) return rc;
  p.src = Y; p.yn = Y; p.acc = A; p.dst = Sa; p.c2 = 0.5 * dt; p.mode = 1;
  if ((rc = batch_stage(b, p, 0, s))) return rc;
  if ((rc = batch_ghosts(b, Sa, s))) return rc;
  p.src = Sa; p.dst = Sb; p.c2 = 0.5 * dt; p.mode = 2;
  if ((rc = batch_stage(b, p, 1, s))) return rc;
  if ((rc = batch_ghosts(b, Sb, s))) return rc;
  p.src = Sb; p.dst = Sa; p.c2 = dt; p.mode = 3;
  if ((rc = batch_stage(b, p, 2, s))) return rc;
  if ((rc = batch_ghosts(b, Sa, s))) return rc;
  p.src = Sa; p.dst = Y; p.c1 = dt / 6.0; p.c2 = 0.0; p.mode = 4;
  return batch_stage(b, p, 3, s);
}

// One RK4 step of patch q with the single-grid kernels.
static int patch_rk4_one(chemora_batch* b, int q, double dt, cudaStream_t s) {
  const PatchDesc& P = b->host_pd[q];
  const int64_t n = b->total;
  double* Y = b->state + P.offset;
  double* A = b->scratch + P.offset;
  double* Sa = b->scratch + n + P.offset;
  double* Sb = b->scratch + 2 * n + P.offset;
  const int kind = b->kind;
  int rc;
  StageParams p{};
  if ((rc = fill_ghosts(P.d, b->nvars, Y, s))) return rc;
  p.src = Y; p.yn = Y; p.acc = A; p.dst = Sa; p.c2 = 0.5 * dt; p.mode = 1;
  if ((rc = launch_stage(kind, P.d, b->sc, p, s))) return rc;
  if ((rc = fill_ghosts(P.d, b->nvars, Sa, s))) return rc;
  p.src = Sa; p.dst = Sb; p.c2 = 0.5 * dt; p.mode = 2;
  if ((rc = launch_stage(kind, P.d, b->sc, p, s))) return rc;
  if ((rc = fill_ghosts(P.d, b->nvars, Sb, s))) return rc;
  p.src = Sb; p.dst = Sa; p.c2 = dt; p.mode = 3;
  if ((rc = launch_stage(kind, P.d, b->sc, p, s))) return rc;
  if ((rc = fill_ghosts(P.d, b->nvars, Sa, s))) return rc;
  p.src = Sa; p.dst = Y; p.c1 = dt / 6.0; p.c2 = 0.0; p.mode = 4;
  return launch_stage(kind, P.d, b->sc, p, s);
}

static void free_graph(chemora_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void destroy_batch(chemora_batch* b) {
  free_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaFree(b->state);
  cudaFree(b->scratch);
  cudaFree(b->dev_pd);
  cudaFree(b->items);
  cudaFree(b->counters);
  cudaFree(b->err);
  b->type = 0;
  delete b;
}

// Capture one batched RK4 step into a graph.  Capture runs on a private
// stream (the legacy default stream cannot be captured); the graph is then
// launched on the caller's stream.
static int capture_step(chemora_batch* b, double dt) {
  free_graph(b);
  if (!b->cap_stream) CHEMORA_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  cudaStream_t s = b->cap_stream;
  CHEMORA_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = batch_rk4_one(b, dt, s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  b->graph = g;
  CHEMORA_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
  b->graph_dt = dt;
  b->graph_kernels = 8;
  return CHEMORA_OK;
}

}  // namespace chemora

using namespace chemora;

extern "C" {

int chemora_patches_create(int npatch, const int* dims, int nghost, double dx, int kind,
                           const chemora_params* params, chemora_batch** out) {
  if (!out) return set_error(CHEMORA_EINVAL, "out is NULL");
  *out = nullptr;
  if (npatch < 1 || !dims) return set_error(CHEMORA_EINVAL, "need npatch >= 1 and dims");
  if (kind != CHEMORA_BSSN && kind != CHEMORA_WAVE)
    return set_error(CHEMORA_EINVAL, "batched patches support CHEMORA_BSSN and CHEMORA_WAVE");
  const int nvars = kind == CHEMORA_BSSN ? 24 : 2;
  if (!(dx > 0.0) || !isfinite(dx)) return set_error(CHEMORA_EINVAL, "dx must be finite and > 0");
  chemora_params prm = {0.1, 2.0, 0, 0, 0};
  if (params) prm = *params;
  if (effective_order(kind, prm) != 4)
    return set_error(CHEMORA_EINVAL, "batched patches use 4th-order differencing");
  int rc = validate_system(kind, nvars, nghost, 4);
  if (rc) return rc;
  if (prm.slicing < 0 || prm.slicing > 2 || prm.shift < 0 || prm.shift > 1)
    return set_error(CHEMORA_EINVAL, "bad params");
  std::vector<PatchDesc> pd(npatch);
  std::vector<WorkItem> items;
  int64_t off = 0;
  for (int q = 0; q < npatch; ++q) {
    const int nx = dims[3 * q], ny = dims[3 * q + 1], nz = dims[3 * q + 2];
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096)
      return set_error(CHEMORA_EINVAL, "patch %d has dims %d x %d x %d (each must be in [1, 4096])",
                       q, nx, ny, nz);
    PatchDesc& P = pd[q];
    const int64_t px = nx + 2 * nghost, py = ny + 2 * nghost, pz = nz + 2 * nghost;
    P.d.nx = nx; P.d.ny = ny; P.d.nz = nz; P.d.g = nghost;
    P.d.sy = px; P.d.sz = px * py; P.d.sv = px * py * pz;
    P.offset = off;
    P.npts = (int64_t)nx * ny * nz;
    off += (P.d.sv * nvars + 31) / 32 * 32;  // 256-byte aligned patch states
    append_items(items, q, P.npts);
  }
  if (items.size() > (size_t)0x7fffffff) return set_error(CHEMORA_EINVAL, "too many work items");
  chemora_batch* b = new (std::nothrow) chemora_batch();
  if (!b) return set_error(CHEMORA_ENOMEM, "host allocation");
  b->type = H_BATCH;
  b->kind = kind; b->nvars = nvars; b->npatch = npatch; b->nghost = nghost; b->dx = dx;
  b->sc = make_scalars(dx, prm);
  b->host_pd = pd;
  b->total = off;
  b->nitems = (int)items.size();
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&b->state, off * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->scratch, 3 * off * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->dev_pd, npatch * sizeof(PatchDesc));
  if (e == cudaSuccess) e = cudaMalloc(&b->items, items.size() * sizeof(WorkItem));
  if (e == cudaSuccess) e = cudaMalloc(&b->counters, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&b->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->state, 0, off * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(b->scratch, 0, 3 * off * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->dev_pd, pd.data(), npatch * sizeof(PatchDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_batch(b);
    return set_error(e == cudaErrorMemoryAllocation ? CHEMORA_ENOMEM : CHEMORA_ECUDA,
                     "batch storage: %s", cudaGetErrorString(e));
  }
  *out = b;
  return CHEMORA_OK;
}

int chemora_patches_inject_fault(chemora_batch* batch, int item) {
  if (!is_handle(batch, H_BATCH)) return set_error(CHEMORA_EINVAL, "not a batch handle");
  if (item < 0 || item >= batch->nitems)
    return set_error(CHEMORA_EINVAL, "work item %d outside [0, %d)", item, batch->nitems);
  const WorkItem bad{batch->npatch + 7, 0};  // names a patch outside the table
  CHEMORA_CUDA(cudaMemcpy(batch->items + item, &bad, sizeof bad, cudaMemcpyHostToDevice));
  return CHEMORA_OK;
}

int chemora_patches_state(chemora_batch* batch, int p, double** dev_ptr) {
  if (!is_handle(batch, H_BATCH)) return set_error(CHEMORA_EINVAL, "not a batch handle");
  if (p < 0 || p >= batch->npatch || !dev_ptr)
    return set_error(CHEMORA_EINVAL, "patch index %d outside [0, %d) or NULL output", p, batch->npatch);
  *dev_ptr = batch->state + batch->host_pd[p].offset;
  return CHEMORA_OK;
}

int chemora_patches_step(chemora_batch* b, double dt, int nsteps, int mode, void* stream) {
  if (!is_handle(b, H_BATCH)) return set_error(CHEMORA_EINVAL, "not a batch handle");
  if (mode != 0 && mode != 1) return set_error(CHEMORA_EINVAL, "mode must be 0 or 1");
  if (nsteps < 0 || !isfinite(dt)) return set_error(CHEMORA_EINVAL, "bad nsteps or dt");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if (mode == 1) {
    for (int n = 0; n < nsteps; ++n)
      for (int q = 0; q < b->npatch; ++q)
        if ((rc = patch_rk4_one(b, q, dt, s))) return rc;
    for (int q = 0; q < b->npatch; ++q)
      if ((rc = fill_ghosts(b->host_pd[q].d, b->nvars, b->state + b->host_pd[q].offset, s))) return rc;
    return CHEMORA_OK;
  }
  cudaStreamCaptureStatus cst;
  CHEMORA_CUDA(cudaStreamIsCapturing(s, &cst));
  if (cst != cudaStreamCaptureStatusNone)
    return set_error(CHEMORA_EINVAL, "chemora_patches_step mode 0 on a stream that is capturing");
  if (!b->exec || b->graph_dt != dt)
    if ((rc = capture_step(b, dt))) return rc;
  for (int n = 0; n < nsteps; ++n) {
    CHEMORA_CUDA(cudaGraphLaunch(b->exec, s));
    if ((rc = launched("cudaGraphLaunch(batched RK4 step)", b->graph_kernels))) return rc;
  }
  if ((rc = batch_ghosts(b, b->state, s))) return rc;
  int herr = 0;
  CHEMORA_CUDA(cudaMemcpyAsync(&herr, b->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CHEMORA_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    cudaMemsetAsync(b->err, 0, sizeof(int), s);
    if (herr & 1) return set_error(CHEMORA_EINVAL, "batched kernel met a work item outside the patch table");
    return set_error(CHEMORA_ETIMEOUT, "a persistent stage launch passed its time limit of %lld SM cycles; "
                     "the batch state is undefined", b->limit_cycles);
  }
  return CHEMORA_OK;
}

int chemora_patches_set_time_limit(chemora_batch* b, double seconds) {
  if (!is_handle(b, H_BATCH)) return set_error(CHEMORA_EINVAL, "not a batch handle");
  if (!isfinite(seconds)) return set_error(CHEMORA_EINVAL, "time limit must be finite");
  long long cycles = 0;
  if (seconds > 0.0) {
    int dev = 0, khz = 0;
    CHEMORA_CUDA(cudaGetDevice(&dev));
    CHEMORA_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const double c = seconds * (double)(khz > 0 ? khz : 2070000) * 1e3;
    cycles = c < 1.0 ? 1 : (c > 9.0e18 ? (long long)9e18 : (long long)c);
  }
  if (cycles != b->limit_cycles) {
    b->limit_cycles = cycles;
    free_graph(b);  // the limit is a kernel argument of the captured step
  }
  return CHEMORA_OK;
}


}  // extern "C"
