// Two-level mesh refinement with Berger-Oliger subcycling for the scalar
// wave (Sec. 4: the Carpet driver refines patches and subcycles them in
// time).  Level 0 is a periodic grid of spacing H; level 1 refines the box
// of coarse points [lo, hi) by 2.  The fine level carries a buffer of
// kBuf = 8 points (stencil radius 2 x 4 RK stages) that prolongation fills
// at the start of every fine step; the RK stages run on the fine interior
// extended by kBuf - 2 points, so the interior stays valid without any
// prolongation at intermediate stages.
//
// Prolongation: quintic Lagrange interpolation along each axis (weights
// 3, -25, 150, 150, -25, 3 over 256 between coarse points, injection at
// coincident ones), applied separably -- x, then y, then z -- to a linear
// combination of coarse time levels (cubic Hermite through y_n, k_n,
// y_{n+1}, k_{n+1}, k the coarse right-hand side).  Restriction: injection
// at coincident points.
#include <math.h>
#include <string.h>

#include <new>

#include "internal.h"

namespace chemora {

constexpr int kBuf = 8;   // fine buffer width
constexpr int kCg = 2;    // coarse ghosts
constexpr int kMargin = 6;  // coarse points the prolongation reads beyond the box

}  // namespace chemora

struct chemora_amr {
  uint32_t type;
  int nc, lo[3], hi[3], nf[3];
  double H;
  chemora::Dims dc;      // coarse grid (ghosts 2)
  chemora::Dims de;      // fine grid seen by the stage kernels: interior + 6, ghosts 2
  chemora::Scalars scc, scf;
  int rc[3], rf[3];      // coarse region and fine padded extents of the prolongation
  double* coarse;        // 2 grid functions (caller-visible)
  double* fine;          // 2 grid functions, padded by kBuf (caller-visible)
  double* cscratch;      // coarse RK scratch: 3 states
  double* fscratch;      // fine RK scratch: 3 states
  double* yn;            // coarse state at t_n
  double* kn;            // coarse RHS at t_n
  double* kn1;           // coarse RHS at t_{n+1}
  double* tcomb;         // time-combined coarse region: 2 x rc^3
  double* ax;            // after the x pass: 2 x rcz x rcy x rfx
  double* axy;           // after the y pass: 2 x rcz x rfy x rfx
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

// tcomb[v][cz][cy][cx] = sum_q w_q C_q at coarse point (lo - 6 + c)
__global__ void amr_time_combine_kernel(Dims dc, int3 lo, int3 rc, TimeLevels tl, double* __restrict__ out) {
  const int64_t n = (int64_t)rc.x * rc.y * rc.z;
  const int v = blockIdx.y;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int cx = (int)(t % rc.x), cy = (int)((t / rc.x) % rc.y), cz = (int)(t / ((int64_t)rc.x * rc.y));
    const int64_t p = (int64_t)(lo.z - kMargin + cz + dc.g) * dc.sz + (int64_t)(lo.y - kMargin + cy + dc.g) * dc.sy +
                      (lo.x - kMargin + cx + dc.g) + v * dc.sv;
    out[v * n + t] = tl.w[0] * tl.c[0][p] + tl.w[1] * tl.c[1][p] + tl.w[2] * tl.c[2][p] + tl.w[3] * tl.c[3][p];
  }
}

// One separable interpolation pass along `axis` (0 x, 1 y, 2 z).  in has
// extents (n0 fastest, n1, n2) with the interpolated axis in coarse-region
// coordinates; out has that axis in fine padded coordinates (size rf).
// For the z pass only fine buffer points are written (into `fine`).
__global__ void amr_prolong_pass_kernel(int axis, const double* __restrict__ in, int3 nin, double* __restrict__ out,
                                        int3 nout, int lo_axis, int3 nf, int64_t fsy, int64_t fsz, int64_t fsv) {
  const int64_t n = (int64_t)nout.x * nout.y * nout.z;
  const int v = blockIdx.y;
  const int64_t nin_t = (int64_t)nin.x * nin.y * nin.z;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    int o[3] = {(int)(t % nout.x), (int)((t / nout.x) % nout.y), (int)(t / ((int64_t)nout.x * nout.y))};
    if (axis == 2) {  // skip fine interior points
      if (o[0] >= kBuf && o[0] < kBuf + nf.x && o[1] >= kBuf && o[1] < kBuf + nf.y && o[2] >= kBuf &&
          o[2] < kBuf + nf.z)
        continue;
    }
    const int F = 2 * lo_axis + (o[axis] - kBuf);  // global fine index along the axis
    int base;
    double w[6];
    const int nw = prolong_weights(F, &base, w);
    const int c0 = base - (lo_axis - kMargin);  // coarse-region coordinate
    int ii[3] = {o[0], o[1], o[2]};
    double s = 0.0;
    for (int q = 0; q < nw; ++q) {
      ii[axis] = c0 + q;
      s += w[q] * in[v * nin_t + ((int64_t)ii[2] * nin.y + ii[1]) * nin.x + ii[0]];
    }
    if (axis == 2)
      out[v * fsv + (int64_t)o[2] * fsz + (int64_t)o[1] * fsy + o[0]] = s;
    else
      out[v * n + t] = s;
  }
}

// coarse[K][J][I] = fine[2(K-lo)+8][2(J-lo)+8][2(I-lo)+8] on the box
__global__ void amr_restrict_kernel(Dims dc, int3 lo, int3 hi, const double* __restrict__ fine, int64_t fsy,
                                    int64_t fsz, int64_t fsv, double* __restrict__ coarse) {
  const int3 n = make_int3(hi.x - lo.x, hi.y - lo.y, hi.z - lo.z);
  const int64_t tot = (int64_t)n.x * n.y * n.z;
  const int v = blockIdx.y;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t % n.x), b = (int)((t / n.x) % n.y), c = (int)(t / ((int64_t)n.x * n.y));
    const int64_t pc = v * dc.sv + (int64_t)(lo.z + c + dc.g) * dc.sz + (int64_t)(lo.y + b + dc.g) * dc.sy +
                       (lo.x + a + dc.g);
    const int64_t pf = v * fsv + (int64_t)(2 * c + kBuf) * fsz + (int64_t)(2 * b + kBuf) * fsy + (2 * a + kBuf);
    coarse[pc] = fine[pf];
  }
}

static int nblocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

// Fill the fine buffer from the coarse time levels with weights w.
static int amr_prolong(chemora_amr* A, const TimeLevels& tl, cudaStream_t s) {
  const int3 lo = make_int3(A->lo[0], A->lo[1], A->lo[2]);
  const int3 rc = make_int3(A->rc[0], A->rc[1], A->rc[2]);
  const int3 rf = make_int3(A->rf[0], A->rf[1], A->rf[2]);
  const int3 nf = make_int3(A->nf[0], A->nf[1], A->nf[2]);
  const int64_t fsy = rf.x, fsz = (int64_t)rf.x * rf.y, fsv = fsz * rf.z;
  int rc_ = CHEMORA_OK;
  const int64_t nt = (int64_t)rc.x * rc.y * rc.z;
  amr_time_combine_kernel<<<dim3(nblocks(nt), 2), 256, 0, s>>>(A->dc, lo, rc, tl, A->tcomb);
  if ((rc_ = launched("amr_time_combine_kernel"))) return rc_;
  const int3 n1 = make_int3(rf.x, rc.y, rc.z);
  amr_prolong_pass_kernel<<<dim3(nblocks((int64_t)n1.x * n1.y * n1.z), 2), 256, 0, s>>>(
      0, A->tcomb, rc, A->ax, n1, lo.x, nf, fsy, fsz, fsv);
  if ((rc_ = launched("amr_prolong_pass_kernel"))) return rc_;
  const int3 n2 = make_int3(rf.x, rf.y, rc.z);
  amr_prolong_pass_kernel<<<dim3(nblocks((int64_t)n2.x * n2.y * n2.z), 2), 256, 0, s>>>(
      1, A->ax, n1, A->axy, n2, lo.y, nf, fsy, fsz, fsv);
  if ((rc_ = launched("amr_prolong_pass_kernel"))) return rc_;
  amr_prolong_pass_kernel<<<dim3(nblocks(fsv), 2), 256, 0, s>>>(2, A->axy, n2, A->fine, rf, lo.z, nf, fsy, fsz,
                                                                fsv);
  return launched("amr_prolong_pass_kernel");
}

// One RK4 step on grid d (buffers y in place, scratch of 3 states).
static int rk4_plain(int kind, const Dims& d, const Scalars& sc, double* Y, double* scratch, double dt,
                     bool ghosts, cudaStream_t s) {
  const size_t n = 2 * (size_t)d.sv;
  double* A = scratch;
  double* Sa = scratch + n;
  double* Sb = scratch + 2 * n;
  double* srcs[4] = {Y, Sa, Sb, Sa};
  double* dsts[4] = {Sa, Sb, Sa, Y};
  const double c2[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  int rc;
  for (int q = 0; q < 4; ++q) {
    if (ghosts && (rc = fill_ghosts(d, 2, srcs[q], s))) return rc;
    StageParams p{};
    p.src = srcs[q]; p.yn = Y; p.acc = A; p.dst = dsts[q];
    p.c1 = dt / 6.0; p.c2 = c2[q]; p.mode = q + 1;
    if ((rc = launch_stage(kind, d, sc, p, s))) return rc;
  }
  return ghosts ? fill_ghosts(d, 2, Y, s) : CHEMORA_OK;
}

}  // namespace chemora

using namespace chemora;

extern "C" {

int chemora_amr_create(int nc, const int* lo, const int* hi, double dx, chemora_amr** out) {
  if (!out) return set_error(CHEMORA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!lo || !hi) return set_error(CHEMORA_EINVAL, "NULL box");
  if (nc < 1 || nc > 4096 || !(dx > 0.0) || !isfinite(dx)) return set_error(CHEMORA_EINVAL, "bad nc or dx");
  for (int d = 0; d < 3; ++d)
    if (lo[d] < 4 || hi[d] > nc - 5 || hi[d] <= lo[d])
      return set_error(CHEMORA_EINVAL,
                       "fine box axis %d is [%d, %d); it must satisfy 4 <= lo < hi <= nc - 5 = %d", d, lo[d],
                       hi[d], nc - 5);
  chemora_amr* A = new (std::nothrow) chemora_amr();
  if (!A) return set_error(CHEMORA_ENOMEM, "host allocation");
  A->type = H_AMR;
  A->nc = nc;
  A->H = dx;
  for (int d = 0; d < 3; ++d) {
    A->lo[d] = lo[d];
    A->hi[d] = hi[d];
    A->nf[d] = 2 * (hi[d] - lo[d]);
    A->rc[d] = hi[d] - lo[d] + 2 * kMargin + 1;
    A->rf[d] = A->nf[d] + 2 * kBuf;
  }
  const int64_t pc = nc + 2 * kCg;
  A->dc = Dims{nc, nc, nc, kCg, pc, pc * pc, pc * pc * pc};
  const int64_t fx = A->rf[0], fy = A->rf[1], fz = A->rf[2];
  A->de = Dims{A->nf[0] + 2 * (kBuf - 2), A->nf[1] + 2 * (kBuf - 2), A->nf[2] + 2 * (kBuf - 2), 2, fx, fx * fy,
               fx * fy * fz};
  chemora_params p = {0.1, 2.0, 0, 0, 0};
  A->scc = make_scalars(dx, p);
  A->scf = make_scalars(0.5 * dx, p);
  const size_t cs = 2 * (size_t)A->dc.sv, fs = 2 * (size_t)A->de.sv;
  const size_t rcn = (size_t)A->rc[0] * A->rc[1] * A->rc[2];
  const size_t axn = (size_t)A->rf[0] * A->rc[1] * A->rc[2];
  const size_t axyn = (size_t)A->rf[0] * A->rf[1] * A->rc[2];
  const size_t total = cs * (1 + 3 + 3) + fs * (1 + 3) + 2 * (rcn + axn + axyn);
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, total * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(buf, 0, total * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (buf) cudaFree(buf);
    delete A;
    return set_error(CHEMORA_ENOMEM, "AMR storage: %s", cudaGetErrorString(e));
  }
  double* q = buf;
  A->coarse = q; q += cs;
  A->cscratch = q; q += 3 * cs;
  A->yn = q; q += cs;
  A->kn = q; q += cs;
  A->kn1 = q; q += cs;
  A->fine = q; q += fs;
  A->fscratch = q; q += 3 * fs;
  A->tcomb = q; q += 2 * rcn;
  A->ax = q; q += 2 * axn;
  A->axy = q;
  *out = A;
  return CHEMORA_OK;
}

int chemora_amr_state(chemora_amr* A, int level, double** dev_ptr, int64_t* sy, int64_t* sz, int64_t* svar) {
  if (!is_handle(A, H_AMR)) return set_error(CHEMORA_EINVAL, "not an AMR handle");
  if (level != 0 && level != 1) return set_error(CHEMORA_EINVAL, "level must be 0 or 1");
  const Dims& d = level == 0 ? A->dc : A->de;
  if (dev_ptr) *dev_ptr = level == 0 ? A->coarse : A->fine;
  if (sy) *sy = d.sy;
  if (sz) *sz = d.sz;
  if (svar) *svar = d.sv;
  return CHEMORA_OK;
}

int chemora_amr_step(chemora_amr* A, double dt, int nsteps, void* stream) {
  if (!is_handle(A, H_AMR)) return set_error(CHEMORA_EINVAL, "not an AMR handle");
  if (nsteps < 0 || !isfinite(dt)) return set_error(CHEMORA_EINVAL, "bad nsteps or dt");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cs = 2 * (size_t)A->dc.sv;
  int rc;
  for (int n = 0; n < nsteps; ++n) {
    if ((rc = fill_ghosts(A->dc, 2, A->coarse, s))) return rc;
    CHEMORA_CUDA(cudaMemcpyAsync(A->yn, A->coarse, cs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    StageParams p{};
    p.src = A->yn; p.dst = A->kn; p.mode = 0;
    if ((rc = launch_stage(CHEMORA_WAVE, A->dc, A->scc, p, s))) return rc;
    if ((rc = fill_ghosts(A->dc, 2, A->kn, s))) return rc;  // read near the box edge
    if ((rc = rk4_plain(CHEMORA_WAVE, A->dc, A->scc, A->coarse, A->cscratch, dt, true, s))) return rc;
    p.src = A->coarse; p.dst = A->kn1;
    if ((rc = launch_stage(CHEMORA_WAVE, A->dc, A->scc, p, s))) return rc;
    if ((rc = fill_ghosts(A->dc, 2, A->kn1, s))) return rc;
    for (int m = 0; m < 2; ++m) {
      const double th = 0.5 * m;
      TimeLevels tl;
      tl.c[0] = A->yn; tl.c[1] = A->kn; tl.c[2] = A->coarse; tl.c[3] = A->kn1;
      tl.w[0] = 2 * th * th * th - 3 * th * th + 1;
      tl.w[1] = dt * (th * th * th - 2 * th * th + th);
      tl.w[2] = -2 * th * th * th + 3 * th * th;
      tl.w[3] = dt * (th * th * th - th * th);
      if ((rc = amr_prolong(A, tl, s))) return rc;
      if ((rc = rk4_plain(CHEMORA_WAVE, A->de, A->scf, A->fine, A->fscratch, 0.5 * dt, false, s))) return rc;
    }
    const int3 lo = make_int3(A->lo[0], A->lo[1], A->lo[2]), hi = make_int3(A->hi[0], A->hi[1], A->hi[2]);
    const int64_t nbox = (int64_t)(hi.x - lo.x) * (hi.y - lo.y) * (hi.z - lo.z);
    amr_restrict_kernel<<<dim3(nblocks(nbox), 2), 256, 0, s>>>(A->dc, lo, hi, A->fine, A->de.sy, A->de.sz,
                                                               A->de.sv, A->coarse);
    if ((rc = launched("amr_restrict_kernel"))) return rc;
  }
  return fill_ghosts(A->dc, 2, A->coarse, s);
}

}  // extern "C"

namespace chemora {
void destroy_amr(chemora_amr* A) {
  cudaFree(A->coarse);  // one allocation, starting at coarse
  A->type = 0;
  delete A;
}
}  // namespace chemora
