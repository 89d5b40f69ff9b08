// RK4 steps of the order-4 scalar wave (Sec. 3, Eq. 1, two-variable form)
// on small grids as a chain of stage kernels joined by programmatic
// dependent launches.
//
// On a 32^3 grid (32,768 points) a graph-replayed RK4 step of the per-stage
// kernels is 8 nodes -- 4 ghost fills, 4 stages -- of about 3 us each, set by
// launch latency rather than by arithmetic.  Here the stage kernel reads
// every neighbour at its periodic image (so no ghost fill is needed between
// stages; the ghosts are filled once per call), and each stage is launched
// as a programmatic dependent launch: the next stage's grid is scheduled
// while the current one runs, and waits in hardware (griddepcontrol.wait)
// until its predecessor has completed and its writes are visible.  Steps are
// captured K at a time in a CUDA graph.  The arithmetic is the generated
// point body and the RK update of the per-stage kernels, so both paths give
// the same bits.  No kernel here spins on memory.
#include <math.h>

#include <new>
#include <vector>

#include "internal.h"
#include "generated/gen_wave.cuh"

namespace chemora {

// Neighbours at their periodic images: offsets of the wrapped x, y and z
// indices (d = -2..2) in the padded layout, read through L2 (the grid may
// start while its predecessor still runs, so nothing is read before the
// dependency wait and nothing is served from the SM's L1).
struct WrapLoader {
  const double* p;  // variable 0 at the padded origin
  int64_t sv;
  int ox[5], oy[5], oz[5];
  __device__ __forceinline__ double operator()(int v, int dx, int dy, int dz) const {
    return __ldcg(p + v * sv + (int64_t)ox[dx + 2] + oy[dy + 2] + oz[dz + 2]);
  }
};

// The scalar wave's fused RK update of StageOutFma (same operations in the
// same order) with y_n and the accumulator of both variables loaded up
// front, together with the neighbours, and the results stored to L2.
struct ChainStageOut {
  const StageParams& a;
  int64_t c, sv;
  double one, two;
  double yn[2], acc[2];
  __device__ __forceinline__ void operator()(int v, double k) const {
    const int64_t cv = c + v * sv;
    switch (a.mode) {
      case 1:
        __stcg(a.acc + cv, k);
        __stcg(a.dst + cv, __fma_rn(a.c2, k, yn[v]));
        break;
      case 2:
      case 3:
        __stcg(a.acc + cv, __fma_rn(two, k, acc[v]));
        __stcg(a.dst + cv, __fma_rn(a.c2, k, yn[v]));
        break;
      default:
        __stcg(a.dst + cv, __fma_rn(a.c1, __fma_rn(acc[v], one, k), yn[v]));
        break;
    }
  }
};

__device__ __forceinline__ int wrap_index(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// One stage (mode 1..4) of the order-4 scalar wave on the interior, one
// point per thread (thread t of block b: interior point 128 b + t, x
// fastest).
__global__ void __launch_bounds__(128) wave_chain_stage_kernel(Dims d, Scalars sc, StageParams a) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int64_t t = (int64_t)blockIdx.x * 128 + threadIdx.x;
  const int64_t npts = (int64_t)d.nx * d.ny * d.nz;
  const int i = (int)(t % d.nx);
  const int j = (int)((t / d.nx) % d.ny);
  const int k = (int)(t / ((int64_t)d.nx * d.ny));
  WrapLoader ld;
  ld.p = a.src;
  ld.sv = d.sv;
#pragma unroll
  for (int m = -2; m <= 2; ++m) {
    ld.ox[m + 2] = wrap_index(i + m, d.nx) + d.g;
    ld.oy[m + 2] = (wrap_index(j + m, d.ny) + d.g) * (int)d.sy;
    ld.oz[m + 2] = (wrap_index(k + m, d.nz) + d.g) * (int)d.sz;
  }
  const int64_t c = (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (t >= npts) return;
  ChainStageOut out{a, c, d.sv, sc.k[CHEMORA_K_ONE], sc.k[CHEMORA_K_TWO], {0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    out.yn[v] = __ldcg(a.yn + c + v * d.sv);
    if (a.mode >= 2) out.acc[v] = __ldcg(a.acc + c + v * d.sv);
  }
  chemora_wave_point(ld, sc, out);
}

struct ChainGraph {
  cudaGraphExec_t exec = nullptr;
  double* state = nullptr;
  double dt = 0.0;
  int steps = 0;
};

// Per-system state: graphs of K steps and of the remainder.
struct ChainState {
  ChainGraph graph[2];
};

constexpr int kChainGraphSteps = 8;

static int chain_stage(const chemora_system* sys, const StageParams& p, cudaStream_t s) {
  const Dims& d = sys->grid->d;
  const int64_t npts = (int64_t)d.nx * d.ny * d.nz;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((npts + 127) / 128));
  cfg.blockDim = dim3(128);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CHEMORA_CUDA(cudaLaunchKernelEx(&cfg, wave_chain_stage_kernel, d, sys->sc, p));
  return launched("wave_chain_stage_kernel");
}

static int chain_steps(const chemora_system* sys, double* Y, double dt, int nsteps, cudaStream_t s) {
  const size_t n = (size_t)sys->nvars * sys->grid->fsize;
  double* acc = sys->scratch;
  double* Sa = sys->scratch + n;
  double* Sb = sys->scratch + 2 * n;
  double* srcs[4] = {Y, Sa, Sb, Sa};
  double* dsts[4] = {Sa, Sb, Sa, Y};
  const double c2[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  int rc;
  for (int step = 0; step < nsteps; ++step)
    for (int q = 0; q < 4; ++q) {
      StageParams p{};
      p.src = srcs[q]; p.yn = Y; p.acc = acc; p.dst = dsts[q];
      p.c1 = dt / 6.0; p.c2 = c2[q]; p.mode = q + 1;
      if ((rc = chain_stage(sys, p, s))) return rc;
    }
  return CHEMORA_OK;
}

static int chain_graph(chemora_system* sys, ChainGraph& g, double* Y, double dt, int steps) {
  if (g.exec && g.state == Y && g.dt == dt && g.steps == steps) return CHEMORA_OK;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  if (!sys->cap_stream) CHEMORA_CUDA(cudaStreamCreateWithFlags(&sys->cap_stream, cudaStreamNonBlocking));
  CHEMORA_CUDA(cudaStreamBeginCapture(sys->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = chain_steps(sys, Y, dt, steps, sys->cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(sys->cap_stream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
  g.state = Y;
  g.dt = dt;
  g.steps = steps;
  return CHEMORA_OK;
}

bool chain_available(const chemora_system* sys) {
  const Dims& d = sys->grid->d;
  // one point per thread in one grid; int offsets
  return sys->kind == CHEMORA_WAVE && sys->sc.order == 4 && d.g >= 2 && d.nx >= 2 && d.ny >= 2 && d.nz >= 2 &&
         (double)d.sv * sys->nvars < 2.0e9 && (double)d.nx * d.ny * d.nz <= 128.0 * 2147483647.0;
}

int chain_rk4(chemora_system* sys, double* state, double dt, int nsteps, cudaStream_t s) {
  if (!chain_available(sys)) return set_error(CHEMORA_EUNSUPPORTED, "no launch-chained step for this system");
  if (!sys->chain) {
    ChainState* cs = new (std::nothrow) ChainState();
    if (!cs) return set_error(CHEMORA_ENOMEM, "host allocation");
    sys->chain = cs;
  }
  ChainState* cs = static_cast<ChainState*>(sys->chain);
  int rc;
  const int full = nsteps / kChainGraphSteps, rest = nsteps % kChainGraphSteps;
  if (full) {
    if ((rc = chain_graph(sys, cs->graph[0], state, dt, kChainGraphSteps))) return rc;
    for (int q = 0; q < full; ++q) {
      CHEMORA_CUDA(cudaGraphLaunch(cs->graph[0].exec, s));
      if ((rc = launched("cudaGraphLaunch(chained RK4 steps)", 4 * kChainGraphSteps))) return rc;
    }
  }
  if (rest) {
    if ((rc = chain_graph(sys, cs->graph[1], state, dt, rest))) return rc;
    CHEMORA_CUDA(cudaGraphLaunch(cs->graph[1].exec, s));
    if ((rc = launched("cudaGraphLaunch(chained RK4 steps)", 4 * rest))) return rc;
  }
  return fill_ghosts(sys->grid->d, sys->nvars, state, s);
}

void chain_free(chemora_system* sys) {
  if (!sys->chain) return;
  ChainState* cs = static_cast<ChainState*>(sys->chain);
  for (ChainGraph& g : cs->graph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  delete cs;
  sys->chain = nullptr;
}

}  // namespace chemora
