// Discrete adjoint of the variable-speed wave equation under RK4: the exact
// transpose of the fully discrete map (the reverse-mode counterpart of the
// Jacobians Kranc generates, Sec. 3.2.1), hand-written.
//
// Forward:  u_t = rho,  rho_t = s Lap u + sum_d G_d D_d u,  G_d = D_d s,
//           s = c^2 (G_d computed once per call; periodic ghosts).
// Transpose of one right-hand side at a stage state y_q, for the cotangent
// kb = (kb_u, kb_rho) of its output, with w = kb_rho:
//   yhat_u   = Lap(s w) - sum_d D_d(G_d w)      (D_d^T = -D_d, Lap^T = Lap)
//   yhat_rho = kb_u
//   sbar    += w Lap u_q - sum_d D_d(w D_d u_q)
// Reverse RK4 step (stage 4 down to 1), from ybar' = cotangent of y_{n+1}:
//   kb_4 = dt/6 ybar';  yhat_q = J^T kb_q;  ybar_n = ybar' + sum_q yhat_q;
//   kb_3 = dt/3 ybar' + dt yhat_4;  kb_2 = dt/3 ybar' + dt/2 yhat_3;
//   kb_1 = dt/6 ybar' + dt/2 yhat_2.
// Checkpoints: y_n every ckpt_every steps.  Each segment but the newest is
// recomputed from its checkpoint with the forward kernel writing a tape
// (Lap u_q and D_d u_q for every stage), so the transpose kernel needs no
// derivatives of u; the newest segment's tape is written by the forward
// pass itself.
//
// Every product is formed at the neighbour points and then differenced, the
// same order as the oracle's definition; a point is written by one thread,
// so results are deterministic.
#include <math.h>
#include <string.h>

#include <vector>

#include "internal.h"

namespace chemora {

constexpr int ATX = 32, ATY = 8;

// FP64 constants of the stage kernels, passed as a kernel parameter.  Every
// add is issued as fma(b, one, a) and every product as fma(a, b, mzero)
// (mzero = -0.0): both give exactly the add's or the product's result, and
// no operand is an immediate.  On GB300 an fma with register or
// constant-bank operands issues faster than DADD, DMUL or an fma with an
// immediate operand.
struct FmaK {
  double one, mzero, eight, sixteen, two;
};

static FmaK fma_k() { return FmaK{1.0, -0.0, 8.0, 16.0, 2.0}; }

__device__ __forceinline__ int64_t at_(const Dims& d, int i, int j, int k) {
  return (int64_t)(k + d.g) * d.sz + (int64_t)(j + d.g) * d.sy + (i + d.g);
}

// Store v at interior point (i, j, k) (offset c) of a grid function and, when
// `imaged`, also at each of its periodic images in the ghost zones (points
// within g of a face have one image per near face, and edge and corner
// images): the ghost zones are then valid without a fill pass.  Needs
// n >= g on every axis (each ghost point then has exactly one interior
// source), which the host checks before passing imaged = 1.
__device__ __forceinline__ void store_imaged(double* f, const Dims& d, int i, int j, int k, int64_t c, double v,
                                             int imaged) {
  f[c] = v;
  if (!imaged) return;
  const int g = d.g;
  int64_t xs[3] = {0, 0, 0}, ys[3] = {0, 0, 0}, zs[3] = {0, 0, 0};
  int nx = 1, ny = 1, nz = 1;
  if (i < g) xs[nx++] = d.nx;
  if (i >= d.nx - g) xs[nx++] = -d.nx;
  if (j < g) ys[ny++] = (int64_t)d.ny * d.sy;
  if (j >= d.ny - g) ys[ny++] = -(int64_t)d.ny * d.sy;
  if (k < g) zs[nz++] = (int64_t)d.nz * d.sz;
  if (k >= d.nz - g) zs[nz++] = -(int64_t)d.nz * d.sz;
  for (int a = 0; a < nx; ++a)
    for (int b = 0; b < ny; ++b)
      for (int e = 0; e < nz; ++e)
        if (a | b | e) f[c + xs[a] + ys[b] + zs[e]] = v;
}

// G_d = D_d s on the interior (3 grid functions).
__global__ void __launch_bounds__(ATX * ATY) varc_grad_s_kernel(Dims d, double i12h,
                                                                const double* __restrict__ s,
                                                                double* __restrict__ G) {
  const int i = blockIdx.x * ATX + threadIdx.x, j = blockIdx.y * ATY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = at_(d, i, j, k);
  const int64_t st[3] = {1, d.sy, d.sz};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double* p = s + c;
    const double a = p[st[q]] - p[-st[q]];
    const double b = p[2 * st[q]] - p[-2 * st[q]];
    G[q * d.sv + c] = (8.0 * a - b) * i12h;
  }
}

// Forward RK stage of the variable-speed wave equation (modes as in the
// stage kernels), optionally writing the tape: Lap u and D_d u of the stage
// state src.
__global__ void __launch_bounds__(ATX * ATY)
varc_fwd_stage_kernel(Dims d, double i12h, double i12h2, const double* __restrict__ s,
                      const double* __restrict__ G, StageParams a, double* __restrict__ tape, FmaK K,
                      int imaged) {
  const int i = blockIdx.x * ATX + threadIdx.x, j = blockIdx.y * ATY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = at_(d, i, j, k);
  const int64_t st[3] = {1, d.sy, d.sz};
  const double* u = a.src + c;
  const double f0 = u[0];
  double lap = K.mzero, adv = K.mzero, du[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int64_t o = st[q];
    const double up1 = u[o], um1 = u[-o], up2 = u[2 * o], um2 = u[-2 * o];
    // (u+1 - f0) + (u-1 - f0), (u+2 - f0) + (u-2 - f0)
    const double d1 = fma(fma(f0, -K.one, um1), K.one, fma(f0, -K.one, up1));
    const double d2 = fma(fma(f0, -K.one, um2), K.one, fma(f0, -K.one, up2));
    lap = fma(fma(K.sixteen, d1, -d2), i12h2, lap);
    // (8 (u+1 - u-1) - (u+2 - u-2)) / (12 h)
    const double t = fma(K.eight, fma(um1, -K.one, up1), -fma(um2, -K.one, up2));
    du[q] = fma(t, i12h, K.mzero);
    adv = fma(G[q * d.sv + c], du[q], adv);
  }
  const double krho = fma(s[c], lap, adv);
  const double ku = a.src[d.sv + c];
  const double kk[2] = {ku, krho};
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    const int64_t cv = c + v * d.sv;
    const double k_ = kk[v];
    // the scalar-wave systems' RK update, each product contracted into its
    // addition (as StageOutFma in the other wave kernels)
    switch (a.mode) {
      case 1:  // acc = k; dst = yn + c2 k
        a.acc[cv] = k_;
        store_imaged(a.dst, d, i, j, k, cv, fma(a.c2, k_, a.yn[cv]), imaged);
        break;
      case 2:
      case 3:  // acc += 2 k; dst = yn + c2 k
        a.acc[cv] = fma(K.two, k_, a.acc[cv]);
        store_imaged(a.dst, d, i, j, k, cv, fma(a.c2, k_, a.yn[cv]), imaged);
        break;
      default:  // dst = yn + c1 (acc + k)
        store_imaged(a.dst, d, i, j, k, cv, fma(a.c1, fma(a.acc[cv], K.one, k_), a.yn[cv]), imaged);
        break;
    }
  }
  if (tape) {
    tape[c] = lap;  // read at the point only
    // D_d u_q is read at stencil neighbours by the transposed stage
    store_imaged(tape, d, i, j, k, d.sv + c, du[0], imaged);
    store_imaged(tape, d, i, j, k, 2 * d.sv + c, du[1], imaged);
    store_imaged(tape, d, i, j, k, 3 * d.sv + c, du[2], imaged);
  }
}

// One transposed stage (see the file comment).  kb: 2 grid functions with
// valid ghosts; tape: Lap u_q (interior) and D_d u_q (ghosts valid).
// first: yacc = yp + yhat (else yacc += yhat).  kbn (if non-NULL):
// kbn = cq yp + aq yhat.
__global__ void __launch_bounds__(ATX * ATY)
varc_adj_stage_kernel(Dims d, double i12h, double i12h2, const double* __restrict__ kb,
                      const double* __restrict__ s, const double* __restrict__ G,
                      const double* __restrict__ tape, const double* __restrict__ yp,
                      double* __restrict__ yacc, double* __restrict__ kbn, double* __restrict__ sbar,
                      double cq, double aq, int first, FmaK K, int imaged) {
  const int i = blockIdx.x * ATX + threadIdx.x, j = blockIdx.y * ATY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = at_(d, i, j, k);
  const int64_t st[3] = {1, d.sy, d.sz};
  const double* w = kb + d.sv + c;  // kb_rho
  const double* sp = s + c;
  const double t0 = fma(sp[0], w[0], K.mzero);
  double lap_sw = K.mzero, div1 = K.mzero, div2 = K.mzero;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int64_t o = st[q];
    const double wp1 = w[o], wm1 = w[-o], wp2 = w[2 * o], wm2 = w[-2 * o];
    // Lap(s w): second differences of the product s w from the centre, each
    // neighbour's product minus the centre's in one fma
    const double d1 = fma(fma(sp[-o], wm1, -t0), K.one, fma(sp[o], wp1, -t0));
    const double d2 = fma(fma(sp[-2 * o], wm2, -t0), K.one, fma(sp[2 * o], wp2, -t0));
    lap_sw = fma(fma(K.sixteen, d1, -d2), i12h2, lap_sw);
    // D_d(G_d w): (8 (p+1 - p-1) - (p+2 - p-2)) / (12 h), p = G_d w
    const double* g = G + q * d.sv + c;
    const double g1 = fma(g[o], wp1, -fma(g[-o], wm1, K.mzero));
    const double g2 = fma(g[2 * o], wp2, -fma(g[-2 * o], wm2, K.mzero));
    div1 = fma(fma(K.eight, g1, -g2), i12h, div1);
    // D_d(w D_d u_q), the same with p = w D_d u_q
    const double* pu = tape + (1 + q) * d.sv + c;
    const double h1 = fma(wp1, pu[o], -fma(wm1, pu[-o], K.mzero));
    const double h2 = fma(wp2, pu[2 * o], -fma(wm2, pu[-2 * o], K.mzero));
    div2 = fma(fma(K.eight, h1, -h2), i12h, div2);
  }
  const double yh[2] = {fma(div1, -K.one, lap_sw), kb[c]};
  sbar[c] = fma(fma(w[0], tape[c], -div2), K.one, sbar[c]);
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    const int64_t cv = c + v * d.sv;
    yacc[cv] = fma(yh[v], K.one, first ? yp[cv] : yacc[cv]);
    if (kbn)  // the next transposed stage reads kb at stencil neighbours
      store_imaged(kbn, d, i, j, k, cv, fma(fma(aq, yh[v], K.mzero), K.one, fma(cq, yp[cv], K.mzero)), imaged);
  }
}

// kb = w ybar' (both components, interior; with its ghost images when imaged)
__global__ void scale_state_kernel(Dims d, double w, const double* __restrict__ y, double* __restrict__ out,
                                   int imaged) {
  const int i = blockIdx.x * ATX + threadIdx.x, j = blockIdx.y * ATY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = at_(d, i, j, k);
  store_imaged(out, d, i, j, k, c, __dmul_rn(w, y[c]), imaged);
  store_imaged(out, d, i, j, k, d.sv + c, __dmul_rn(w, y[d.sv + c]), imaged);
}

// Loss J = 1/2 sum (u[r] - data_r)^2 and the seed ybar_u[r] += u[r] - data_r.
// One block; a fixed tree reduction keeps the loss deterministic.
__global__ void receivers_kernel(const double* __restrict__ u, const int64_t* __restrict__ recv,
                                 const double* __restrict__ data, int nrecv, double* ybar_u,
                                 double* loss) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int r = threadIdx.x; r < nrecv; r += blockDim.x) {
    const double m = u[recv[r]] - data[r];
    acc += 0.5 * m * m;
    atomicAdd(ybar_u + recv[r], m);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0];
}

// grad_c = 2 c sbar on the interior, ghosts of grad_c zero.
__global__ void grad_c_kernel(Dims d, const double* __restrict__ c, const double* __restrict__ sbar,
                              double* __restrict__ gc) {
  const int i = blockIdx.x * ATX + threadIdx.x, j = blockIdx.y * ATY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t p = at_(d, i, j, k);
  gc[p] = 2.0 * c[p] * sbar[p];
}

// s = c^2 on the interior
__global__ void adj_square_kernel(Dims d, const double* __restrict__ c, double* __restrict__ s) {
  const int i = blockIdx.x * ATX + threadIdx.x, j = blockIdx.y * ATY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t p = at_(d, i, j, k);
  s[p] = c[p] * c[p];
}

// out = in on the interior of nv grid functions
__global__ void copy_interior_kernel(Dims d, int nv, const double* __restrict__ in, double* __restrict__ out) {
  const int i = blockIdx.x * ATX + threadIdx.x, j = blockIdx.y * ATY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t p = at_(d, i, j, k);
  for (int v = 0; v < nv; ++v) out[v * d.sv + p] = in[v * d.sv + p];
}

static dim3 agrid(const Dims& d) { return dim3((d.nx + ATX - 1) / ATX, (d.ny + ATY - 1) / ATY, d.nz); }

int launch_varc_grad(const Dims& d, double i12h, const double* s, double* G, cudaStream_t st) {
  varc_grad_s_kernel<<<agrid(d), dim3(ATX, ATY), 0, st>>>(d, i12h, s, G);
  return launched("varc_grad_s_kernel");
}

struct AdjBufs {
  double *s, *G, *Y, *ck, *seg, *tape, *yp, *yacc, *kb, *kbn, *sbar, *loss;
  int64_t* recv;
  double* data;
};

// One forward RK4 step of the variable-speed wave (in place on Y), tape of
// the 4 stages written at tape (16 grid functions) when non-NULL.
// Stage outputs written with their ghost images (no fill passes) when every
// axis has at least g points.
static int imaged_ok(const Dims& d) { return d.nx >= d.g && d.ny >= d.g && d.nz >= d.g ? 1 : 0; }

static int fwd_step(chemora_system* sys, const AdjBufs& B, double* Y, double dt, double* tape,
                    cudaStream_t s) {
  const Dims& d = sys->grid->d;
  const int im = imaged_ok(d);
  const size_t fs = sys->grid->fsize;
  double* A = sys->scratch;
  double* Sa = sys->scratch + 2 * fs;
  double* Sb = sys->scratch + 4 * fs;
  const double i12h = sys->sc.i12h, i12h2 = sys->sc.i12h2;
  StageParams p{};
  int rc;
  double* srcs[4] = {Y, Sa, Sb, Sa};
  double* dsts[4] = {Sa, Sb, Sa, Y};
  const double c2[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  for (int q = 0; q < 4; ++q) {
    if (!im && (rc = fill_ghosts(d, 2, srcs[q], s))) return rc;
    p.src = srcs[q]; p.yn = Y; p.acc = A; p.dst = dsts[q]; p.c1 = dt / 6.0; p.c2 = c2[q]; p.mode = q + 1;
    varc_fwd_stage_kernel<<<agrid(d), dim3(ATX, ATY), 0, s>>>(d, i12h, i12h2, B.s, B.G, p,
                                                                tape ? tape + (size_t)q * 4 * fs : nullptr,
                                                                fma_k(), im);
    if ((rc = launched("varc_fwd_stage_kernel"))) return rc;
  }
  return im ? CHEMORA_OK : fill_ghosts(d, 2, Y, s);
}

// One reverse RK4 step: on entry B.yp holds ybar'; on exit B.yacc holds ybar_n.
static int rev_step(chemora_system* sys, const AdjBufs& B, const double* tape, double dt, cudaStream_t s) {
  const Dims& d = sys->grid->d;
  const size_t fs = sys->grid->fsize;
  const double i12h = sys->sc.i12h, i12h2 = sys->sc.i12h2;
  const int im = imaged_ok(d);
  int rc;
  scale_state_kernel<<<agrid(d), dim3(ATX, ATY), 0, s>>>(d, dt / 6.0, B.yp, B.kb, im);
  if ((rc = launched("scale_state_kernel"))) return rc;
  const double cq[4] = {0.0, dt / 6.0, dt / 3.0, dt / 3.0};  // weight of ybar' in kb_{q-1}
  const double aq[4] = {0.0, 0.5 * dt, 0.5 * dt, dt};        // a_q dt
  double* kb = B.kb;
  double* kbn = B.kbn;
  for (int q = 3; q >= 0; --q) {
    if (!im && (rc = fill_ghosts(d, 2, kb, s))) return rc;
    varc_adj_stage_kernel<<<agrid(d), dim3(ATX, ATY), 0, s>>>(
        d, i12h, i12h2, kb, B.s, B.G, tape + (size_t)q * 4 * fs, B.yp, B.yacc, q > 0 ? kbn : nullptr,
        B.sbar, cq[q], aq[q], q == 3 ? 1 : 0, fma_k(), im);
    if ((rc = launched("varc_adj_stage_kernel"))) return rc;
    double* t = kb;
    kb = kbn;
    kbn = t;
  }
  return CHEMORA_OK;
}

}  // namespace chemora

using namespace chemora;

extern "C" int chemora_adjoint_rk4(chemora_system* sys, const double* state0, const double* c,
                                   double dt, int nsteps, int ckpt_every, const int64_t* recv_idx,
                                   int nrecv, const double* data, double* loss, double* grad_state0,
                                   double* grad_c, void* stream) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (sys->kind != CHEMORA_WAVE_VARC)
    return set_error(CHEMORA_EINVAL, "chemora_adjoint_rk4 needs a CHEMORA_WAVE_VARC system");
  if (!state0 || !c || !recv_idx || !data || !loss || !grad_state0 || !grad_c)
    return set_error(CHEMORA_EINVAL, "NULL argument");
  if (nsteps < 1 || ckpt_every < 1 || nrecv < 1 || !isfinite(dt))
    return set_error(CHEMORA_EINVAL, "need nsteps >= 1, ckpt_every >= 1, nrecv >= 1, finite dt");
  const Dims& d = sys->grid->d;
  const size_t fs = sys->grid->fsize;
  for (int r = 0; r < nrecv; ++r) {
    const int64_t p = recv_idx[r];
    if (p < 0 || p >= (int64_t)fs) return set_error(CHEMORA_EINVAL, "receiver %d outside the grid", r);
    const int64_t k = p / d.sz, j = (p % d.sz) / d.sy, i = p % d.sy;
    if (i < d.g || i >= d.g + d.nx || j < d.g || j >= d.g + d.ny || k < d.g || k >= d.g + d.nz)
      return set_error(CHEMORA_EINVAL, "receiver %d (index %lld) is not an interior point", r,
                       (long long)p);
  }
  int rc = ensure_scratch(sys);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int K = ckpt_every < nsteps ? ckpt_every : nsteps;
  const int nck = (nsteps + K - 1) / K;
  // fields: s 1, G 3, Y 2, ck 2 nck, seg 2 K, tape 16 K, yp 2, yacc 2, kb 2, kbn 2, sbar 1, loss
  const size_t nfields = 1 + 3 + 2 + 2 * (size_t)nck + 2 * (size_t)K + 16 * (size_t)K + 2 + 2 + 2 + 2 + 1;
  const size_t bytes = (nfields * fs + 32) * sizeof(double) + (size_t)nrecv * (sizeof(int64_t) + sizeof(double));
  char* buf = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&buf, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(CHEMORA_ENOMEM, "adjoint work space of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  AdjBufs B;
  double* q = (double*)buf;
  B.s = q; q += fs;
  B.G = q; q += 3 * fs;
  B.Y = q; q += 2 * fs;
  B.ck = q; q += 2 * (size_t)nck * fs;
  B.seg = q; q += 2 * (size_t)K * fs;
  B.tape = q; q += 16 * (size_t)K * fs;
  B.yp = q; q += 2 * fs;
  B.yacc = q; q += 2 * fs;
  B.kb = q; q += 2 * fs;
  B.kbn = q; q += 2 * fs;
  B.sbar = q; q += fs;
  B.loss = q; q += 32;
  B.recv = (int64_t*)q;
  B.data = (double*)(B.recv + nrecv);

  auto run = [&]() -> int {
    int r;
    CHEMORA_CUDA(cudaMemsetAsync(B.yp, 0, 2 * fs * sizeof(double), s));
    CHEMORA_CUDA(cudaMemsetAsync(B.sbar, 0, fs * sizeof(double), s));
    CHEMORA_CUDA(cudaMemcpyAsync(B.recv, recv_idx, nrecv * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CHEMORA_CUDA(cudaMemcpyAsync(B.data, data, nrecv * sizeof(double), cudaMemcpyHostToDevice, s));
    // s = c^2 with ghosts; G = D s with ghosts
    adj_square_kernel<<<agrid(d), dim3(ATX, ATY), 0, s>>>(d, c, B.s);
    if ((r = launched("adj_square_kernel"))) return r;
    if ((r = fill_ghosts(d, 1, B.s, s))) return r;
    if ((r = launch_varc_grad(d, sys->sc.i12h, B.s, B.G, s))) return r;
    if ((r = fill_ghosts(d, 3, B.G, s))) return r;
    // forward pass with checkpoints; the newest segment's steps write their
    // tape here (the same kernel on the same states as a recomputation), so
    // the reverse sweep recomputes only the older segments
    const int nlast = (nck - 1) * K;
    CHEMORA_CUDA(cudaMemcpyAsync(B.Y, state0, 2 * fs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if ((r = fill_ghosts(d, 2, B.Y, s))) return r;
    for (int n = 0; n < nsteps; ++n) {
      if (n % K == 0)
        CHEMORA_CUDA(cudaMemcpyAsync(B.ck + (size_t)(n / K) * 2 * fs, B.Y, 2 * fs * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
      double* tp = n >= nlast ? B.tape + (size_t)(n - nlast) * 16 * fs : nullptr;
      if ((r = fwd_step(sys, B, B.Y, dt, tp, s))) return r;
    }
    // loss and seed
    receivers_kernel<<<1, 1024, 0, s>>>(B.Y, B.recv, B.data, nrecv, B.yp, B.loss);
    if ((r = launched("receivers_kernel"))) return r;
    // reverse sweep, newest segment first
    for (int sg = nck - 1; sg >= 0; --sg) {
      const int n0 = sg * K, n1 = (n0 + K < nsteps) ? n0 + K : nsteps;
      if (sg < nck - 1)
        CHEMORA_CUDA(cudaMemcpyAsync(B.seg, B.ck + (size_t)sg * 2 * fs, 2 * fs * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
      for (int n = n0; n < n1 && sg < nck - 1; ++n) {
        double* yn = B.seg + (size_t)(n - n0) * 2 * fs;
        if (n + 1 < n1) {
          double* y1 = yn + 2 * fs;
          CHEMORA_CUDA(cudaMemcpyAsync(y1, yn, 2 * fs * sizeof(double), cudaMemcpyDeviceToDevice, s));
          if ((r = fwd_step(sys, B, y1, dt, B.tape + (size_t)(n - n0) * 16 * fs, s))) return r;
        } else {
          // last step of the segment: only its tape is needed
          CHEMORA_CUDA(cudaMemcpyAsync(B.Y, yn, 2 * fs * sizeof(double), cudaMemcpyDeviceToDevice, s));
          if ((r = fwd_step(sys, B, B.Y, dt, B.tape + (size_t)(n - n0) * 16 * fs, s))) return r;
        }
      }
      // the tape's D_d u fields are read at stencil neighbours: periodic
      // ghosts (written with their images by the forward kernel when it can)
      if (!imaged_ok(d) && (r = fill_ghosts(d, 16 * (n1 - n0), B.tape, s))) return r;
      for (int n = n1 - 1; n >= n0; --n) {
        if ((r = rev_step(sys, B, B.tape + (size_t)(n - n0) * 16 * fs, dt, s))) return r;
        double* t = B.yp;
        B.yp = B.yacc;
        B.yacc = t;
      }
    }
    // outputs
    CHEMORA_CUDA(cudaMemsetAsync(grad_state0, 0, 2 * fs * sizeof(double), s));
    CHEMORA_CUDA(cudaMemsetAsync(grad_c, 0, fs * sizeof(double), s));
    copy_interior_kernel<<<agrid(d), dim3(ATX, ATY), 0, s>>>(d, 2, B.yp, grad_state0);
    if ((r = launched("copy_interior_kernel"))) return r;
    grad_c_kernel<<<agrid(d), dim3(ATX, ATY), 0, s>>>(d, c, B.sbar, grad_c);
    if ((r = launched("grad_c_kernel"))) return r;
    CHEMORA_CUDA(cudaMemcpyAsync(loss, B.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    return CHEMORA_OK;
  };
  rc = run();
  cudaFreeAsync(buf, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (rc) return rc;
  if (e2 != cudaSuccess) return cuda_error(e2, "cudaStreamSynchronize(adjoint)");
  return CHEMORA_OK;
}
