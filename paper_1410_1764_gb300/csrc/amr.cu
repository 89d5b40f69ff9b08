// Two-level mesh refinement with Berger-Oliger subcycling (Sec. 4: the
// Carpet driver refines patches and subcycles them in time) for the scalar
// wave and the BSSN system, 4th order.  Level 0 is a periodic grid of
// spacing H; level 1 is a set of disjoint boxes, each refining a block of
// coarse points [lo, hi) by 2.  Each box carries a buffer of B = 4 r points
// (r the stencil radius: 2 for the wave, 3 for BSSN, whose dissipation
// stencil reaches 3 points; B = r x 4 RK stages) that prolongation fills at
// the start of every fine step from the coarse level; the RK stages then run
// on the box interior extended into the buffer, stage s on the region whose
// distance from the buffer's outer edge is at least r s, so the interior
// stays valid without any prolongation at intermediate stages and no point
// is computed that a later stage does not read.
//
// The boxes are patches of a batched work-list (the persistent stage kernel
// of patches.cu): one launch per fine RK stage advances every box, over a
// per-stage patch table whose interiors shrink by r per stage.  For
// comparison, mode 1 launches the single-grid stage kernel box by box.
//
// Prolongation: quintic Lagrange interpolation along each axis (weights
// 3, -25, 150, 150, -25, 3 over 256 between coarse points, injection at
// coincident ones), applied separably -- x, then y, then z -- to a linear
// combination of coarse time levels (cubic Hermite through y_n, k_n,
// y_{n+1}, k_{n+1}, k the coarse right-hand side); each pass is one launch
// over every box and variable.  Restriction: injection at coincident
// points, one launch over every box.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

namespace chemora {

struct AmrBox {
  int lo[3], hi[3];
  int nf[3];   // fine interior points per axis: 2 (hi - lo)
  int rc[3];   // coarse region the prolongation reads: [lo - M, hi + M] per axis, M = B/2 + 2
  int rf[3];   // padded fine extents: nf + 2 B
  int64_t fine_off;               // first double of the box's state in the fine storage
  int64_t tc_off, ax_off, axy_off;  // prolongation work arrays (per variable: their region size)
};

}  // namespace chemora

struct chemora_amr {
  uint32_t type;
  int kind, nv;
  int r, B, M, gc;  // stencil radius, buffer, prolongation margin (coarse points), coarse ghosts
  int nc[3];
  double H;
  chemora::Dims dc;  // coarse grid
  chemora::Scalars scc, scf;
  int nbox;
  std::vector<chemora::AmrBox> boxes;
  std::vector<chemora::PatchDesc> stage_pd;  // 4 x nbox: fine stage s (1..4) of box b at (s-1) nbox + b
  int item_off[5];                           // stage s's items: [item_off[s-1], item_off[s])
  int mode;                                  // 0: batched boxes, 1: box by box
  int coarse_variant;                        // launch shape of the coarse stage kernel (chemora_amr_autotune)
  double* coarse;    // nv grid functions (caller-visible)
  double* cscratch;  // coarse RK scratch: 3 states
  double* yn;        // coarse state at t_n
  double* kn;        // coarse RHS at t_n
  double* kn1;       // coarse RHS at t_{n+1}
  double* fine;      // every box's state, padded by B (caller-visible views)
  double* fscratch;  // acc, stage a, stage b of every box: 3 x ftotal
  int64_t ftotal;    // doubles of all box states
  double* pwork;     // prolongation work arrays of every box
  chemora::AmrBox* dev_boxes;
  chemora::PatchDesc* dev_pd;
  chemora::WorkItem* items;
  unsigned int* counters;  // 8: fine step (2) x stage (4) of a coarse step
  int* err;
};

namespace chemora {

__device__ __forceinline__ int prolong_weights(int F, int* base, double* w) {
  if ((F & 1) == 0) {
    *base = F >> 1;
    w[0] = 1.0;
    return 1;
  }
  *base = ((F - 1) >> 1) - 2;
  w[0] = 3.0 / 256.0;
  w[1] = -25.0 / 256.0;
  w[2] = 150.0 / 256.0;
  w[3] = 150.0 / 256.0;
  w[4] = -25.0 / 256.0;
  w[5] = 3.0 / 256.0;
  return 6;
}

struct TimeLevels {
  const double* c[4];
  double w[4];
};

// tcomb of box b, variable v: sum_q w_q C_q at coarse point (lo - M + c);
// blockIdx.y = variable, blockIdx.z = box.
__global__ void amr_time_combine_kernel(Dims dc, const AmrBox* __restrict__ boxes, int M, TimeLevels tl,
                                        double* __restrict__ work) {
  const AmrBox& bx = boxes[blockIdx.z];
  const int3 rc = make_int3(bx.rc[0], bx.rc[1], bx.rc[2]);
  const int64_t n = (int64_t)rc.x * rc.y * rc.z;
  const int v = blockIdx.y;
  double* out = work + bx.tc_off + v * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int cx = (int)(t % rc.x), cy = (int)((t / rc.x) % rc.y), cz = (int)(t / ((int64_t)rc.x * rc.y));
    const int64_t p = (int64_t)(bx.lo[2] - M + cz + dc.g) * dc.sz + (int64_t)(bx.lo[1] - M + cy + dc.g) * dc.sy +
                      (bx.lo[0] - M + cx + dc.g) + v * dc.sv;
    out[t] = tl.w[0] * tl.c[0][p] + tl.w[1] * tl.c[1][p] + tl.w[2] * tl.c[2][p] + tl.w[3] * tl.c[3][p];
  }
}

// One separable interpolation pass along `axis` (0 x, 1 y, 2 z) of every
// box (blockIdx.z) and variable (blockIdx.y).  Pass x reads tcomb (rc.x,
// rc.y, rc.z) and writes ax (rf.x, rc.y, rc.z); pass y writes axy (rf.x,
// rf.y, rc.z); pass z writes the buffer points of the box state (rf.x,
// rf.y, rf.z), leaving its interior alone.
__global__ void amr_prolong_pass_kernel(int axis, const AmrBox* __restrict__ boxes, int B, int M, int nv,
                                        double* work, double* __restrict__ fine) {
  const AmrBox& bx = boxes[blockIdx.z];
  const int v = blockIdx.y;
  int3 nin, nout;
  const double* in;
  if (axis == 0) {
    nin = make_int3(bx.rc[0], bx.rc[1], bx.rc[2]);
    nout = make_int3(bx.rf[0], bx.rc[1], bx.rc[2]);
    in = work + bx.tc_off;
  } else if (axis == 1) {
    nin = make_int3(bx.rf[0], bx.rc[1], bx.rc[2]);
    nout = make_int3(bx.rf[0], bx.rf[1], bx.rc[2]);
    in = work + bx.ax_off;
  } else {
    nin = make_int3(bx.rf[0], bx.rf[1], bx.rc[2]);
    nout = make_int3(bx.rf[0], bx.rf[1], bx.rf[2]);
    in = work + bx.axy_off;
  }
  const int64_t n = (int64_t)nout.x * nout.y * nout.z;
  const int64_t nin_t = (int64_t)nin.x * nin.y * nin.z;
  in += v * nin_t;
  const int lo_axis = bx.lo[axis];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    int o[3] = {(int)(t % nout.x), (int)((t / nout.x) % nout.y), (int)(t / ((int64_t)nout.x * nout.y))};
    if (axis == 2) {  // skip fine interior points
      if (o[0] >= B && o[0] < B + bx.nf[0] && o[1] >= B && o[1] < B + bx.nf[1] && o[2] >= B &&
          o[2] < B + bx.nf[2])
        continue;
    }
    const int F = 2 * lo_axis + (o[axis] - B);  // global fine index along the axis
    int base;
    double w[6];
    const int nw = prolong_weights(F, &base, w);
    const int c0 = base - (lo_axis - M);  // coarse-region coordinate
    int ii[3] = {o[0], o[1], o[2]};
    double s = 0.0;
    for (int q = 0; q < nw; ++q) {
      ii[axis] = c0 + q;
      s += w[q] * in[((int64_t)ii[2] * nin.y + ii[1]) * nin.x + ii[0]];
    }
    if (axis == 2)
      fine[bx.fine_off + v * n + t] = s;
    else
      work[(axis == 0 ? bx.ax_off : bx.axy_off) + v * n + t] = s;
  }
}

// coarse[K][J][I] = fine[2(K-lo)+B][2(J-lo)+B][2(I-lo)+B] on every box
// (blockIdx.z) and variable (blockIdx.y).
__global__ void amr_restrict_kernel(Dims dc, const AmrBox* __restrict__ boxes, int B, const double* __restrict__ fine,
                                    double* __restrict__ coarse) {
  const AmrBox& bx = boxes[blockIdx.z];
  const int3 n = make_int3(bx.hi[0] - bx.lo[0], bx.hi[1] - bx.lo[1], bx.hi[2] - bx.lo[2]);
  const int64_t tot = (int64_t)n.x * n.y * n.z;
  const int64_t fsy = bx.rf[0], fsz = fsy * bx.rf[1], fsv = fsz * bx.rf[2];
  const int v = blockIdx.y;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t % n.x), b = (int)((t / n.x) % n.y), c = (int)(t / ((int64_t)n.x * n.y));
    const int64_t pc = v * dc.sv + (int64_t)(bx.lo[2] + c + dc.g) * dc.sz + (int64_t)(bx.lo[1] + b + dc.g) * dc.sy +
                       (bx.lo[0] + a + dc.g);
    const int64_t pf = bx.fine_off + v * fsv + (int64_t)(2 * c + B) * fsz + (int64_t)(2 * b + B) * fsy + (2 * a + B);
    coarse[pc] = fine[pf];
  }
}

static int nblocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

// Fill every box's buffer from the coarse time levels with weights w.
static int amr_prolong(chemora_amr* A, const TimeLevels& tl, cudaStream_t s) {
  int64_t nt = 0, n1 = 0, n2 = 0, n3 = 0;
  for (const AmrBox& b : A->boxes) {
    nt = std::max<int64_t>(nt, (int64_t)b.rc[0] * b.rc[1] * b.rc[2]);
    n1 = std::max<int64_t>(n1, (int64_t)b.rf[0] * b.rc[1] * b.rc[2]);
    n2 = std::max<int64_t>(n2, (int64_t)b.rf[0] * b.rf[1] * b.rc[2]);
    n3 = std::max<int64_t>(n3, (int64_t)b.rf[0] * b.rf[1] * b.rf[2]);
  }
  int rc;
  amr_time_combine_kernel<<<dim3(nblocks(nt), A->nv, A->nbox), 256, 0, s>>>(A->dc, A->dev_boxes, A->M, tl,
                                                                             A->pwork);
  if ((rc = launched("amr_time_combine_kernel"))) return rc;
  const int64_t np[3] = {n1, n2, n3};
  for (int axis = 0; axis < 3; ++axis) {
    amr_prolong_pass_kernel<<<dim3(nblocks(np[axis]), A->nv, A->nbox), 256, 0, s>>>(
        axis, A->dev_boxes, A->B, A->M, A->nv, A->pwork, A->fine);
    if ((rc = launched("amr_prolong_pass_kernel"))) return rc;
  }
  return CHEMORA_OK;
}

// One RK4 step of the periodic coarse grid (buffers y in place, scratch of 3
// states).  Stage 1's right-hand side k_1 = RHS(y_n) is the coarse time
// level k_n of the prolongation: it is copied out of the accumulator (which
// holds exactly k_1 after stage 1) into kn, ghosts included, instead of
// being evaluated again.
static int rk4_coarse(chemora_amr* A, double* Y, double dt, double* kn, cudaStream_t s) {
  const Dims& d = A->dc;
  const size_t n = (size_t)A->nv * d.sv;
  double* acc = A->cscratch;
  double* Sa = A->cscratch + n;
  double* Sb = A->cscratch + 2 * n;
  double* srcs[4] = {Y, Sa, Sb, Sa};
  double* dsts[4] = {Sa, Sb, Sa, Y};
  const double c2[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  int rc;
  for (int q = 0; q < 4; ++q) {
    if ((rc = fill_ghosts(d, A->nv, srcs[q], s))) return rc;
    StageParams p{};
    p.src = srcs[q]; p.yn = Y; p.acc = acc; p.dst = dsts[q];
    p.c1 = dt / 6.0; p.c2 = c2[q]; p.mode = q + 1;
    if ((rc = launch_stage(A->kind, d, A->scc, p, s, A->coarse_variant))) return rc;
    if (q == 0) {
      CHEMORA_CUDA(cudaMemcpyAsync(kn, acc, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      if ((rc = fill_ghosts(d, A->nv, kn, s))) return rc;  // read near the box edges
    }
  }
  return fill_ghosts(d, A->nv, Y, s);
}

// One RK4 step of dt of every box (buffers prolonged before), stage s over
// the box interior extended by B - r s.  `step` (0 or 1) picks the work-list
// counters of the coarse step's first or second fine step.
static int rk4_fine(chemora_amr* A, double dt, int step, cudaStream_t s) {
  const int64_t n = A->ftotal;
  double* Y = A->fine;
  double* acc = A->fscratch;
  double* Sa = A->fscratch + n;
  double* Sb = A->fscratch + 2 * n;
  double* srcs[4] = {Y, Sa, Sb, Sa};
  double* dsts[4] = {Sa, Sb, Sa, Y};
  const double c2[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  int rc;
  for (int q = 0; q < 4; ++q) {
    StageParams p{};
    p.src = srcs[q]; p.yn = Y; p.acc = acc; p.dst = dsts[q];
    p.c1 = dt / 6.0; p.c2 = c2[q]; p.mode = q + 1;
    if (A->mode == 0) {
      const int i0 = A->item_off[q], i1 = A->item_off[q + 1];
      if ((rc = launch_batch_stage(A->nv, A->dev_pd + q * A->nbox, A->nbox, A->items + i0, i1 - i0,
                                   A->counters + 4 * step + q, A->err, 0, A->scf, p, s)))
        return rc;
    } else {
      for (int b = 0; b < A->nbox; ++b) {
        const PatchDesc& P = A->stage_pd[q * A->nbox + b];
        StageParams pb = p;
        pb.src += P.offset; pb.yn += P.offset; pb.acc += P.offset; pb.dst += P.offset;
        if ((rc = launch_stage(A->kind, P.d, A->scf, pb, s))) return rc;
      }
    }
  }
  return CHEMORA_OK;
}

static int create_amr(int kind, const int* nc, int nbox, const int* lo, const int* hi, double dx,
                      const chemora_params* params, chemora_amr** out) {
  if (!out) return set_error(CHEMORA_EINVAL, "out is NULL");
  *out = nullptr;
  if (kind != CHEMORA_WAVE && kind != CHEMORA_BSSN)
    return set_error(CHEMORA_EINVAL, "mesh refinement supports CHEMORA_WAVE and CHEMORA_BSSN");
  if (!nc || !lo || !hi) return set_error(CHEMORA_EINVAL, "NULL extents or boxes");
  if (nbox < 1 || nbox > 4096) return set_error(CHEMORA_EINVAL, "need 1 <= nbox <= 4096 (got %d)", nbox);
  if (!(dx > 0.0) || !isfinite(dx)) return set_error(CHEMORA_EINVAL, "dx must be finite and > 0");
  chemora_params prm = {0.1, 2.0, 0, 0, 0};
  if (params) prm = *params;
  if (effective_order(kind, prm) != 4) return set_error(CHEMORA_EINVAL, "mesh refinement uses 4th-order differencing");
  if (prm.slicing < 0 || prm.slicing > 2 || prm.shift < 0 || prm.shift > 1 || !isfinite(prm.eps_diss) ||
      !isfinite(prm.eta))
    return set_error(CHEMORA_EINVAL, "bad params");
  const int r = kind == CHEMORA_BSSN ? 3 : 2, B = 4 * r, M = B / 2 + 2, gc = r;
  for (int d = 0; d < 3; ++d)
    if (nc[d] < 1 || nc[d] > 4096) return set_error(CHEMORA_EINVAL, "coarse extent %d on axis %d", nc[d], d);
  for (int b = 0; b < nbox; ++b)
    for (int d = 0; d < 3; ++d) {
      const int l = lo[3 * b + d], h = hi[3 * b + d];
      if (l < M - gc || h > nc[d] + gc - 1 - M || h <= l)
        return set_error(CHEMORA_EINVAL,
                         "box %d axis %d is [%d, %d); it must satisfy %d <= lo < hi <= %d (the prolongation of "
                         "its %d-point buffer reads %d coarse points beyond the box)",
                         b, d, l, h, M - gc, nc[d] + gc - 1 - M, B, M);
    }
  for (int a = 0; a < nbox; ++a)
    for (int b = a + 1; b < nbox; ++b) {
      bool overlap = true;
      for (int d = 0; d < 3; ++d)
        if (hi[3 * a + d] <= lo[3 * b + d] || hi[3 * b + d] <= lo[3 * a + d]) overlap = false;
      if (overlap) return set_error(CHEMORA_EINVAL, "boxes %d and %d overlap", a, b);
    }
  const int nv = kind == CHEMORA_BSSN ? 24 : 2;
  chemora_amr* A = new (std::nothrow) chemora_amr();
  if (!A) return set_error(CHEMORA_ENOMEM, "host allocation");
  A->type = H_AMR;
  A->kind = kind; A->nv = nv; A->r = r; A->B = B; A->M = M; A->gc = gc;
  A->H = dx;
  A->nbox = nbox;
  for (int d = 0; d < 3; ++d) A->nc[d] = nc[d];
  const int64_t px = nc[0] + 2 * gc, py = nc[1] + 2 * gc, pz = nc[2] + 2 * gc;
  A->dc = Dims{nc[0], nc[1], nc[2], gc, px, px * py, px * py * pz};
  A->scc = make_scalars(dx, prm);
  A->scf = make_scalars(0.5 * dx, prm);
  // boxes: state offsets (256-byte aligned) and prolongation work arrays
  int64_t foff = 0, woff = 0;
  A->boxes.resize(nbox);
  for (int b = 0; b < nbox; ++b) {
    AmrBox& X = A->boxes[b];
    for (int d = 0; d < 3; ++d) {
      X.lo[d] = lo[3 * b + d];
      X.hi[d] = hi[3 * b + d];
      X.nf[d] = 2 * (X.hi[d] - X.lo[d]);
      X.rc[d] = X.hi[d] - X.lo[d] + 2 * M + 1;
      X.rf[d] = X.nf[d] + 2 * B;
    }
    const int64_t fsv = (int64_t)X.rf[0] * X.rf[1] * X.rf[2];
    X.fine_off = foff;
    foff += (nv * fsv + 31) / 32 * 32;
    X.tc_off = woff;
    woff += (int64_t)nv * X.rc[0] * X.rc[1] * X.rc[2];
    X.ax_off = woff;
    woff += (int64_t)nv * X.rf[0] * X.rc[1] * X.rc[2];
    X.axy_off = woff;
    woff += (int64_t)nv * X.rf[0] * X.rf[1] * X.rc[2];
  }
  A->ftotal = foff;
  // fine stage tables: stage s (1..4) computes the interior extended by B - r s
  std::vector<WorkItem> items;
  A->stage_pd.resize(4 * nbox);
  A->item_off[0] = 0;
  for (int q = 0; q < 4; ++q) {
    const int g = r * (q + 1);
    for (int b = 0; b < nbox; ++b) {
      const AmrBox& X = A->boxes[b];
      PatchDesc& P = A->stage_pd[q * nbox + b];
      const int64_t sy = X.rf[0], sz = sy * X.rf[1], sv = sz * X.rf[2];
      P.d = Dims{X.rf[0] - 2 * g, X.rf[1] - 2 * g, X.rf[2] - 2 * g, g, sy, sz, sv};
      P.offset = X.fine_off;
      P.npts = (int64_t)P.d.nx * P.d.ny * P.d.nz;
      append_items(items, b, P.npts);  // patch index within the stage's table
    }
    if (items.size() > (size_t)0x7fffffff) {
      delete A;
      return set_error(CHEMORA_EINVAL, "too many work items");
    }
    A->item_off[q + 1] = (int)items.size();
  }
  const size_t cs = (size_t)nv * A->dc.sv;
  const size_t total = cs * (1 + 3 + 3) + (size_t)foff * (1 + 3) + (size_t)woff;
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, total * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(buf, 0, total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&A->dev_boxes, nbox * sizeof(AmrBox));
  if (e == cudaSuccess) e = cudaMalloc(&A->dev_pd, 4 * nbox * sizeof(PatchDesc));
  if (e == cudaSuccess) e = cudaMalloc(&A->items, items.size() * sizeof(WorkItem));
  if (e == cudaSuccess) e = cudaMalloc(&A->counters, 8 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&A->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(A->err, 0, sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(A->dev_boxes, A->boxes.data(), nbox * sizeof(AmrBox), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(A->dev_pd, A->stage_pd.data(), 4 * nbox * sizeof(PatchDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(A->items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(buf);
    cudaFree(A->dev_boxes);
    cudaFree(A->dev_pd);
    cudaFree(A->items);
    cudaFree(A->counters);
    cudaFree(A->err);
    delete A;
    return set_error(e == cudaErrorMemoryAllocation ? CHEMORA_ENOMEM : CHEMORA_ECUDA, "AMR storage: %s",
                     cudaGetErrorString(e));
  }
  double* q = buf;
  A->coarse = q; q += cs;
  A->cscratch = q; q += 3 * cs;
  A->yn = q; q += cs;
  A->kn = q; q += cs;
  A->kn1 = q; q += cs;
  A->fine = q; q += foff;
  A->fscratch = q; q += 3 * foff;
  A->pwork = q;
  *out = A;
  return CHEMORA_OK;
}

}  // namespace chemora

using namespace chemora;

extern "C" {

int chemora_amr_create_boxes(int kind, const int* nc, int nbox, const int* lo, const int* hi, double dx,
                             const chemora_params* params, chemora_amr** out) {
  return create_amr(kind, nc, nbox, lo, hi, dx, params, out);
}

int chemora_amr_create(int nc, const int* lo, const int* hi, double dx, chemora_amr** out) {
  const int n3[3] = {nc, nc, nc};
  return create_amr(CHEMORA_WAVE, n3, 1, lo, hi, dx, nullptr, out);
}

int chemora_amr_state(chemora_amr* A, int level, double** dev_ptr, int64_t* sy, int64_t* sz, int64_t* svar) {
  if (!is_handle(A, H_AMR)) return set_error(CHEMORA_EINVAL, "not an AMR handle");
  if (level < 0 || level > A->nbox)
    return set_error(CHEMORA_EINVAL, "level %d outside [0, %d] (0 coarse, 1 + b box b)", level, A->nbox);
  if (level == 0) {
    if (dev_ptr) *dev_ptr = A->coarse;
    if (sy) *sy = A->dc.sy;
    if (sz) *sz = A->dc.sz;
    if (svar) *svar = A->dc.sv;
    return CHEMORA_OK;
  }
  const AmrBox& X = A->boxes[level - 1];
  if (dev_ptr) *dev_ptr = A->fine + X.fine_off;
  if (sy) *sy = X.rf[0];
  if (sz) *sz = (int64_t)X.rf[0] * X.rf[1];
  if (svar) *svar = (int64_t)X.rf[0] * X.rf[1] * X.rf[2];
  return CHEMORA_OK;
}

int chemora_amr_step_mode(chemora_amr* A, double dt, int nsteps, int mode, void* stream) {
  if (!is_handle(A, H_AMR)) return set_error(CHEMORA_EINVAL, "not an AMR handle");
  if (nsteps < 0 || !isfinite(dt)) return set_error(CHEMORA_EINVAL, "bad nsteps or dt");
  if (mode != 0 && mode != 1) return set_error(CHEMORA_EINVAL, "mode must be 0 (batched) or 1 (box by box)");
  A->mode = mode;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cs = (size_t)A->nv * A->dc.sv;
  const int nv = A->nv;
  int rc;
  for (int n = 0; n < nsteps; ++n) {
    if ((rc = fill_ghosts(A->dc, nv, A->coarse, s))) return rc;
    CHEMORA_CUDA(cudaMemcpyAsync(A->yn, A->coarse, cs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if ((rc = rk4_coarse(A, A->coarse, dt, A->kn, s))) return rc;  // also k_n = RHS(y_n)
    StageParams p{};
    p.src = A->coarse; p.dst = A->kn1; p.mode = 0;
    if ((rc = launch_stage(A->kind, A->dc, A->scc, p, s, A->coarse_variant))) return rc;
    if ((rc = fill_ghosts(A->dc, nv, A->kn1, s))) return rc;
    if (mode == 0) CHEMORA_CUDA(cudaMemsetAsync(A->counters, 0, 8 * sizeof(unsigned int), s));
    for (int m = 0; m < 2; ++m) {
      const double th = 0.5 * m;
      TimeLevels tl;
      tl.c[0] = A->yn; tl.c[1] = A->kn; tl.c[2] = A->coarse; tl.c[3] = A->kn1;
      tl.w[0] = 2 * th * th * th - 3 * th * th + 1;
      tl.w[1] = dt * (th * th * th - 2 * th * th + th);
      tl.w[2] = -2 * th * th * th + 3 * th * th;
      tl.w[3] = dt * (th * th * th - th * th);
      if ((rc = amr_prolong(A, tl, s))) return rc;
      if ((rc = rk4_fine(A, 0.5 * dt, m, s))) return rc;
    }
    int64_t nmax = 0;
    for (const AmrBox& X : A->boxes)
      nmax = std::max<int64_t>(nmax, (int64_t)(X.hi[0] - X.lo[0]) * (X.hi[1] - X.lo[1]) * (X.hi[2] - X.lo[2]));
    amr_restrict_kernel<<<dim3(nblocks(nmax), nv, A->nbox), 256, 0, s>>>(A->dc, A->dev_boxes, A->B, A->fine,
                                                                         A->coarse);
    if ((rc = launched("amr_restrict_kernel"))) return rc;
  }
  if ((rc = fill_ghosts(A->dc, nv, A->coarse, s))) return rc;
  if (mode == 0 && nsteps > 0) {
    int herr = 0;
    CHEMORA_CUDA(cudaMemcpyAsync(&herr, A->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CHEMORA_CUDA(cudaStreamSynchronize(s));
    if (herr) {
      cudaMemsetAsync(A->err, 0, sizeof(int), s);
      return set_error(CHEMORA_ECUDA, "batched fine stage reported error word %d", herr);
    }
  }
  return CHEMORA_OK;
}

int chemora_amr_autotune(chemora_amr* A, int* variant, void* stream) {
  if (!is_handle(A, H_AMR)) return set_error(CHEMORA_EINVAL, "not an AMR handle");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if ((rc = fill_ghosts(A->dc, A->nv, A->coarse, s))) return rc;
  const size_t cs = (size_t)A->nv * A->dc.sv;
  StageParams p{};  // a middle RK stage into the coarse scratch
  p.src = A->coarse; p.yn = A->coarse; p.acc = A->cscratch; p.dst = A->cscratch + cs; p.mode = 2;
  int best = A->coarse_variant;
  if ((rc = autotune_stage(A->kind, A->dc, A->scc, p, s, &best, nullptr))) return rc;
  A->coarse_variant = best;
  if (variant) *variant = best;
  return CHEMORA_OK;
}

int chemora_amr_step(chemora_amr* A, double dt, int nsteps, void* stream) {
  return chemora_amr_step_mode(A, dt, nsteps, 0, stream);
}

}  // extern "C"

namespace chemora {
void destroy_amr(chemora_amr* A) {
  cudaFree(A->coarse);  // one allocation, starting at coarse
  cudaFree(A->dev_boxes);
  cudaFree(A->dev_pd);
  cudaFree(A->items);
  cudaFree(A->counters);
  cudaFree(A->err);
  A->type = 0;
  delete A;
}
}  // namespace chemora
