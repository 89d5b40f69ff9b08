/*
 * Chemora hot-path oracle: a plain, slow, FP64 CPU implementation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * What it computes (Chemora, arXiv 1410.1764):
 *   - periodic ghost zones around a uniform Cartesian grid (Sec. 2, driver
 *     ghost zones for domain decomposition);
 *   - 4th-order centred finite-difference operators (Sec. 3.2.2, "standard"
 *     finite differencing of arbitrary order) and 5th-order Kreiss-Oliger
 *     dissipation;
 *   - right-hand sides of the scalar wave equation in first-order-in-time
 *     form (Sec. 3, Eq. 1, two-variable reading), of the variable-speed wave
 *     equation, and of the Einstein equations in BSSN phi-form (the Einstein
 *     equations of Sec. 3.4 and Sec. 5; the paper prints no BSSN formulas, so
 *     the standard phi-form system is written out here term by term);
 *   - the classic 4-stage Runge-Kutta method of lines (Sec. 2, time
 *     integrator thorn);
 *   - the exact discrete transpose of the variable-speed wave step and the
 *     stage-wise reverse of RK4 with checkpoint recomputation.
 *
 * Rounding order: differences of symmetric neighbour pairs (first
 * derivatives) or of neighbours against the centre (second derivatives,
 * dissipation) are formed first, then scaled by a precomputed 1/(12h),
 * 1/(12h^2), 1/(144h^2) or eps/(64h).  Build with -ffp-contract=off.
 *
 * Layout: every grid function is a contiguous array [nz+2g][ny+2g][nx+2g]
 * (x fastest), ghosts included; a state of nv variables is nv such arrays
 * back to back.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nx, ny, nz, g;
  double h;
} orc_grid;

typedef struct {
  double eps_diss; /* Kreiss-Oliger strength */
  double eta;      /* Gamma-driver damping */
  int slicing;     /* 0: 1+log, 1: harmonic, 2: frozen lapse */
  int shift;       /* 0: Gamma-driver, 1: frozen shift (and B) */
  int order;       /* finite-difference order of the wave systems (0 = 4) */
} orc_params;

enum { ORC_WAVE = 1, ORC_WAVE_VARC = 2, ORC_BSSN = 3, ORC_WAVE1 = 4 };

int orc_wave_rhs_order(const double* st, double* rhs, const orc_grid* G, int order);
int orc_wave1_rhs(const double* st, double* rhs, const orc_grid* G, int order);

static size_t px_(const orc_grid* G) { return (size_t)G->nx + 2 * G->g; }
static size_t py_(const orc_grid* G) { return (size_t)G->ny + 2 * G->g; }
static size_t pz_(const orc_grid* G) { return (size_t)G->nz + 2 * G->g; }
static size_t plane_(const orc_grid* G) { return px_(G) * py_(G); }
static size_t fsize_(const orc_grid* G) { return plane_(G) * pz_(G); }

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the later parallel loops (n >= 1); results do not depend on it:
 * every point is computed by one thread from the same inputs. */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* Ghost zones: the value at padded index (i,j,k) is the value at the  */
/* interior point with the same coordinates modulo the period.         */
/* ------------------------------------------------------------------ */
static int wrap_(int i, int n, int g) {
  int r = (i - g) % n;
  if (r < 0) r += n;
  return r + g;
}

void orc_fill_ghosts(double* f, int nvars, const orc_grid* G) {
  const int px = (int)px_(G), py = (int)py_(G), pz = (int)pz_(G), g = G->g;
  const size_t fs = fsize_(G), pl = plane_(G);
  for (int v = 0; v < nvars; ++v) {
    double* a = f + (size_t)v * fs;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < pz; ++k)
      for (int j = 0; j < py; ++j)
        for (int i = 0; i < px; ++i) {
          int interior = i >= g && i < g + G->nx && j >= g && j < g + G->ny &&
                         k >= g && k < g + G->nz;
          if (interior) continue;
          int si = wrap_(i, G->nx, g), sj = wrap_(j, G->ny, g), sk = wrap_(k, G->nz, g);
          a[(size_t)k * pl + (size_t)j * px + i] = a[(size_t)sk * pl + (size_t)sj * px + si];
        }
  }
}

/* ------------------------------------------------------------------ */
/* Stencils (Sec. 3.2.2).  p points at the centre, s is the stride of  */
/* the direction.  The unscaled forms return 12h*D1, 12h^2*D2,         */
/* 144h^2*D11 and 64h/eps*KO respectively.                             */
/* ------------------------------------------------------------------ */
static double st_d1(const double* p, ptrdiff_t s) {
  double a = p[s] - p[-s];
  double b = p[2 * s] - p[-2 * s];
  return 8.0 * a - b;
}
static double st_d2(const double* p, ptrdiff_t s) {
  double f0 = p[0];
  double d1 = (p[s] - f0) + (p[-s] - f0);
  double d2 = (p[2 * s] - f0) + (p[-2 * s] - f0);
  return 16.0 * d1 - d2;
}
static double st_d11(const double* p, ptrdiff_t sa, ptrdiff_t sb) {
  double r[5];
  for (int m = -2; m <= 2; ++m) r[m + 2] = st_d1(p + m * sb, sa);
  double a = r[3] - r[1];
  double b = r[4] - r[0];
  return 8.0 * a - b;
}
static double st_ko(const double* p, ptrdiff_t s) {
  double f0 = p[0];
  double d1 = (p[s] - f0) + (p[-s] - f0);
  double d2 = (p[2 * s] - f0) + (p[-2 * s] - f0);
  double d3 = (p[3 * s] - f0) + (p[-3 * s] - f0);
  return d3 - 6.0 * d2 + 15.0 * d1;
}

/* Derivative field of one grid function on the interior (test access to the
 * stencils).  kind 0: D1 along a; 1: pure D2 along a; 2: mixed D_a D_b;
 * 3: Kreiss-Oliger term along a with eps = 1.  Ghost entries of out are left
 * untouched. */
void orc_deriv(const double* f, double* out, const orc_grid* G, int kind, int a, int b) {
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const double h = G->h;
  const double i12h = 1.0 / (12.0 * h), i12h2 = 1.0 / (12.0 * h * h);
  const double i144h2 = 1.0 / (144.0 * h * h), i64h = 1.0 / (64.0 * h);
  const int g = G->g;
#pragma omp parallel for schedule(static)
  for (int k = g; k < g + G->nz; ++k)
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        const double* p = f + c;
        double r;
        switch (kind) {
          case 0: r = st_d1(p, str[a]) * i12h; break;
          case 1: r = st_d2(p, str[a]) * i12h2; break;
          case 2: r = st_d11(p, str[a], str[b]) * i144h2; break;
          default: r = st_ko(p, str[a]) * i64h; break;
        }
        out[c] = r;
      }
}

/* ------------------------------------------------------------------ */
/* Scalar wave equation, Sec. 3 Eq. (1) in second-order-in-space form:  */
/*   u_t = rho,   rho_t = Laplacian_h u.                               */
/* ------------------------------------------------------------------ */
void orc_wave_rhs(const double* st, double* rhs, const orc_grid* G) {
  const size_t fs = fsize_(G);
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const double i12h2 = 1.0 / (12.0 * G->h * G->h);
  const int g = G->g;
#pragma omp parallel for schedule(static)
  for (int k = g; k < g + G->nz; ++k)
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        const double* u = st + c;
        double lap = st_d2(u, str[0]) * i12h2 + st_d2(u, str[1]) * i12h2 +
                     st_d2(u, str[2]) * i12h2;
        rhs[c] = st[fs + c];
        rhs[fs + c] = lap;
      }
}

/* ------------------------------------------------------------------ */
/* Variable-speed wave equation u_tt = s Lap u + grad s . grad u with   */
/* s = c^2 a grid function (ghosts valid):                              */
/*   u_t = rho,   rho_t = s Lap_h u + sum_d D_d s D_d u.                */
/* ------------------------------------------------------------------ */
void orc_varc_rhs(const double* st, const double* s, double* rhs, const orc_grid* G) {
  const size_t fs = fsize_(G);
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const double i12h = 1.0 / (12.0 * G->h), i12h2 = 1.0 / (12.0 * G->h * G->h);
  const int g = G->g;
#pragma omp parallel for schedule(static)
  for (int k = g; k < g + G->nz; ++k)
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        const double* u = st + c;
        const double* sp = s + c;
        double lap = 0.0, adv = 0.0;
        for (int d = 0; d < 3; ++d) {
          lap += st_d2(u, str[d]) * i12h2;
          adv += (st_d1(sp, str[d]) * i12h) * (st_d1(u, str[d]) * i12h);
        }
        rhs[c] = st[fs + c];
        rhs[fs + c] = s[c] * lap + adv;
      }
}

/* Tangent-linear variable-speed wave right-hand side: the derivative of
 * orc_varc_rhs at (st, s) in the direction (dst, ds):
 *   du_t = drho,  drho_t = s Lap du + sum D s D du + ds Lap u + sum D ds D u. */
void orc_varc_tlm_rhs(const double* st, const double* s, const double* dst, const double* ds,
                      double* drhs, const orc_grid* G) {
  const size_t fs = fsize_(G);
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const double i12h = 1.0 / (12.0 * G->h), i12h2 = 1.0 / (12.0 * G->h * G->h);
  const int g = G->g;
#pragma omp parallel for schedule(static)
  for (int k = g; k < g + G->nz; ++k)
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        double lap_du = 0, lap_u = 0, a1 = 0, a2 = 0;
        for (int d = 0; d < 3; ++d) {
          lap_du += st_d2(dst + c, str[d]) * i12h2;
          lap_u += st_d2(st + c, str[d]) * i12h2;
          a1 += (st_d1(s + c, str[d]) * i12h) * (st_d1(dst + c, str[d]) * i12h);
          a2 += (st_d1(ds + c, str[d]) * i12h) * (st_d1(st + c, str[d]) * i12h);
        }
        drhs[c] = dst[fs + c];
        drhs[fs + c] = s[c] * lap_du + a1 + ds[c] * lap_u + a2;
      }
}

/* Transposed right-hand side of the variable-speed wave equation.  Given the
 * cotangent kb = (kb_u, kb_rho) of a right-hand side evaluated at state st,
 * this returns yhat = J^T kb and accumulates the cotangent of s:
 *   yhat_u   = Lap(s kb_rho) - sum_d D_d (D_d s * kb_rho)
 *   yhat_rho = kb_u
 *   sbar    += kb_rho Lap u - sum_d D_d (kb_rho D_d u)
 * On a periodic grid D_d^T = -D_d and Lap^T = Lap.  Temporary products are
 * formed as periodic grid functions and the stencils applied to them.
 * kb's ghost zones are ignored; yhat's and sbar's ghosts are left alone. */
void orc_varc_adj_rhs(const double* st, const double* s, const double* kb, double* yhat,
                      double* sbar, const orc_grid* G) {
  const size_t fs = fsize_(G);
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const double i12h = 1.0 / (12.0 * G->h), i12h2 = 1.0 / (12.0 * G->h * G->h);
  const int g = G->g;
  /* t[0] = s*kb_rho; t[1..3] = D_d s * kb_rho; t[4..6] = kb_rho * D_d u */
  double* t = (double*)calloc(7 * fs, sizeof(double));
  if (!t) return;
#pragma omp parallel for schedule(static)
  for (int k = g; k < g + G->nz; ++k)
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        double w = kb[fs + c];
        t[c] = s[c] * w;
        for (int d = 0; d < 3; ++d) {
          t[(1 + d) * fs + c] = (st_d1(s + c, str[d]) * i12h) * w;
          t[(4 + d) * fs + c] = w * (st_d1(st + c, str[d]) * i12h);
        }
      }
  orc_fill_ghosts(t, 7, G);
#pragma omp parallel for schedule(static)
  for (int k = g; k < g + G->nz; ++k)
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        double lap_sw = 0, div1 = 0, lap_u = 0, div2 = 0;
        for (int d = 0; d < 3; ++d) {
          lap_sw += st_d2(t + c, str[d]) * i12h2;
          div1 += st_d1(t + (1 + d) * fs + c, str[d]) * i12h;
          lap_u += st_d2(st + c, str[d]) * i12h2;
          div2 += st_d1(t + (4 + d) * fs + c, str[d]) * i12h;
        }
        yhat[c] = lap_sw - div1;
        yhat[fs + c] = kb[c];
        sbar[c] += kb[fs + c] * lap_u - div2;
      }
  free(t);
}

/* ------------------------------------------------------------------ */
/* Einstein equations, BSSN phi-form.  Variable order:                 */
/*  0 phi; 1-6 gt_ij (xx,xy,xz,yy,yz,zz); 7 K; 8-13 At_ij; 14-16 Xt^i; */
/*  17 alpha; 18-20 beta^i; 21-23 B^i.                                  */
/* ------------------------------------------------------------------ */
static const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
/* variables that need second derivatives: phi, gt_ij, alpha, beta^i */
static int needs_dd_(int v) { return v == 0 || (v >= 1 && v <= 6) || v == 17 || (v >= 18 && v <= 20); }

typedef struct {
  double u[24];
  double d[24][3];
  double dd[24][3][3];
  /* derived geometry */
  double gt[3][3], gtu[3][3], At[3][3], Atm[3][3], Atu[3][3];
  double Gl[3][3][3], Gu[3][3][3], Xtn[3];
  double dphi[3], dal[3], dK[3], dgt[3][3][3], dAt[3][3][3], dbe[3][3], dXt[3][3];
  double e4, AA;
} bssn_pt;

static void bssn_load_(const double* st, size_t fs, const ptrdiff_t str[3], size_t c, double h,
                       bssn_pt* P) {
  const double i12h = 1.0 / (12.0 * h), i12h2 = 1.0 / (12.0 * h * h);
  const double i144h2 = 1.0 / (144.0 * h * h);
  for (int v = 0; v < 24; ++v) {
    const double* p = st + (size_t)v * fs + c;
    P->u[v] = p[0];
    for (int a = 0; a < 3; ++a) P->d[v][a] = st_d1(p, str[a]) * i12h;
    if (needs_dd_(v)) {
      for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b) {
          double r = (a == b) ? st_d2(p, str[a]) * i12h2 : st_d11(p, str[a], str[b]) * i144h2;
          P->dd[v][a][b] = r;
          P->dd[v][b][a] = r;
        }
    }
  }
  /* named views */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      P->gt[i][j] = P->u[1 + SYM[i][j]];
      P->At[i][j] = P->u[8 + SYM[i][j]];
      P->dbe[i][j] = P->d[18 + i][j];
      P->dXt[i][j] = P->d[14 + i][j];
      for (int k = 0; k < 3; ++k) {
        P->dgt[i][j][k] = P->d[1 + SYM[i][j]][k];
        P->dAt[i][j][k] = P->d[8 + SYM[i][j]][k];
      }
    }
  for (int k = 0; k < 3; ++k) {
    P->dphi[k] = P->d[0][k];
    P->dal[k] = P->d[17][k];
    P->dK[k] = P->d[7][k];
  }
  /* inverse conformal metric: adjugate over determinant */
  const double (*g)[3] = (const double (*)[3])P->gt;
  double c00 = g[1][1] * g[2][2] - g[1][2] * g[2][1];
  double c01 = g[1][2] * g[2][0] - g[1][0] * g[2][2];
  double c02 = g[1][0] * g[2][1] - g[1][1] * g[2][0];
  double det = g[0][0] * c00 + g[0][1] * c01 + g[0][2] * c02;
  double idet = 1.0 / det;
  P->gtu[0][0] = c00 * idet;
  P->gtu[0][1] = P->gtu[1][0] = (g[0][2] * g[2][1] - g[0][1] * g[2][2]) * idet;
  P->gtu[0][2] = P->gtu[2][0] = (g[0][1] * g[1][2] - g[0][2] * g[1][1]) * idet;
  P->gtu[1][1] = (g[0][0] * g[2][2] - g[0][2] * g[2][0]) * idet;
  P->gtu[1][2] = P->gtu[2][1] = (g[0][2] * g[1][0] - g[0][0] * g[1][2]) * idet;
  P->gtu[2][2] = (g[0][0] * g[1][1] - g[0][1] * g[1][0]) * idet;
  /* Christoffel symbols of the first kind: Gl[k][i][j] = Gamma~_{kij} */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        P->Gl[k][i][j] = 0.5 * (P->dgt[j][k][i] + P->dgt[i][k][j] - P->dgt[i][j][k]);
  /* second kind: Gu[k][i][j] = Gamma~^k_{ij} */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += P->gtu[k][l] * P->Gl[l][i][j];
        P->Gu[k][i][j] = s;
      }
  /* contracted Christoffel Gamma~^k_(d) = gt^{ij} Gamma~^k_{ij} */
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) s += P->gtu[i][j] * P->Gu[k][i][j];
    P->Xtn[k] = s;
  }
  P->e4 = exp(-4.0 * P->u[0]);
  /* At with raised indices */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += P->gtu[i][k] * P->At[k][j];
      P->Atm[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += P->gtu[i][k] * P->gtu[j][l] * P->At[k][l];
      P->Atu[i][j] = s;
    }
  double AA = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) AA += P->At[i][j] * P->Atu[i][j];
  P->AA = AA;
}

/* Ricci tensor R_ij = R~_ij + R^phi_ij and the lapse Hessian D_i D_j alpha. */
static void bssn_ricci_(const bssn_pt* P, double R[3][3], double DDal[3][3], double* trDDal) {
  const double (*gtu)[3] = (const double (*)[3])P->gtu;
  double DDphi[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = P->dd[0][i][j];
      for (int k = 0; k < 3; ++k) s -= P->Gu[k][i][j] * P->dphi[k];
      DDphi[i][j] = s;
    }
  double trDDphi = 0.0, dphi2 = 0.0, dphidal = 0.0, trddal = 0.0, Xdal = 0.0;
  for (int l = 0; l < 3; ++l)
    for (int m = 0; m < 3; ++m) {
      trDDphi += gtu[l][m] * DDphi[l][m];
      dphi2 += gtu[l][m] * P->dphi[l] * P->dphi[m];
      dphidal += gtu[l][m] * P->dphi[l] * P->dal[m];
      trddal += gtu[l][m] * P->dd[17][l][m];
    }
  for (int k = 0; k < 3; ++k) Xdal += P->Xtn[k] * P->dal[k];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      /* conformal Ricci */
      double t1 = 0.0;
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) t1 += gtu[l][m] * P->dd[1 + SYM[i][j]][l][m];
      double t2 = 0.0;
      for (int k = 0; k < 3; ++k) t2 += P->gt[k][i] * P->dXt[k][j] + P->gt[k][j] * P->dXt[k][i];
      double t3 = 0.0;
      for (int k = 0; k < 3; ++k) t3 += P->Xtn[k] * (P->Gl[i][j][k] + P->Gl[j][i][k]);
      double t4 = 0.0;
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          double s = 0.0;
          for (int k = 0; k < 3; ++k)
            s += P->Gu[k][l][i] * P->Gl[j][k][m] + P->Gu[k][l][j] * P->Gl[i][k][m] +
                 P->Gu[k][i][m] * P->Gl[k][l][j];
          t4 += gtu[l][m] * s;
        }
      double Rt = -0.5 * t1 + 0.5 * t2 + 0.5 * t3 + t4;
      /* conformal-factor part */
      double Rphi = -2.0 * DDphi[i][j] - 2.0 * P->gt[i][j] * trDDphi +
                    4.0 * P->dphi[i] * P->dphi[j] - 4.0 * P->gt[i][j] * dphi2;
      R[i][j] = Rt + Rphi;
      /* physical Hessian of the lapse, conformal decomposition */
      double h = P->dd[17][i][j];
      for (int k = 0; k < 3; ++k) h -= P->Gu[k][i][j] * P->dal[k];
      h -= 2.0 * (P->dphi[i] * P->dal[j] + P->dphi[j] * P->dal[i]);
      h += 2.0 * P->gt[i][j] * dphidal;
      DDal[i][j] = h;
    }
  *trDDal = P->e4 * (trddal - Xdal + 2.0 * dphidal);
}

static void bssn_point_rhs_(const bssn_pt* P, const orc_params* prm, double out[24]) {
  const double (*gtu)[3] = (const double (*)[3])P->gtu;
  const double* u = P->u;
  const double al = u[17], K = u[7];
  const double be[3] = {u[18], u[19], u[20]};
  double adv[24];
  for (int v = 0; v < 24; ++v) adv[v] = be[0] * P->d[v][0] + be[1] * P->d[v][1] + be[2] * P->d[v][2];
  double divbe = P->dbe[0][0] + P->dbe[1][1] + P->dbe[2][2];
  double R[3][3], DDal[3][3], trDDal;
  bssn_ricci_(P, R, DDal, &trDDal);

  /* phi */
  out[0] = adv[0] + (divbe - al * K) / 6.0;
  /* gt_ij */
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double s = adv[1 + SYM[i][j]];
      for (int k = 0; k < 3; ++k) s += P->gt[i][k] * P->dbe[k][j] + P->gt[j][k] * P->dbe[k][i];
      s -= (2.0 / 3.0) * P->gt[i][j] * divbe;
      s -= 2.0 * al * P->At[i][j];
      out[1 + SYM[i][j]] = s;
    }
  /* K */
  out[7] = adv[7] - trDDal + al * (P->AA + K * K / 3.0);
  /* At_ij */
  double X[3][3], trX = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X[i][j] = -DDal[i][j] + al * R[i][j];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) trX += gtu[k][l] * X[k][l];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double s = adv[8 + SYM[i][j]];
      for (int k = 0; k < 3; ++k) s += P->At[i][k] * P->dbe[k][j] + P->At[j][k] * P->dbe[k][i];
      s -= (2.0 / 3.0) * P->At[i][j] * divbe;
      s += P->e4 * (X[i][j] - P->gt[i][j] * trX / 3.0);
      double AtAt = 0.0;
      for (int k = 0; k < 3; ++k) AtAt += P->At[i][k] * P->Atm[k][j];
      s += al * (K * P->At[i][j] - 2.0 * AtAt);
      out[8 + SYM[i][j]] = s;
    }
  /* Xt^i */
  double rXt[3];
  for (int i = 0; i < 3; ++i) {
    double s = adv[14 + i];
    for (int j = 0; j < 3; ++j) s -= P->Xtn[j] * P->dbe[i][j];
    s += (2.0 / 3.0) * P->Xtn[i] * divbe;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += gtu[j][k] * P->dd[18 + i][j][k];
    for (int j = 0; j < 3; ++j) {
      double ddb = 0.0;
      for (int k = 0; k < 3; ++k) ddb += P->dd[18 + k][j][k];
      s += gtu[i][j] * ddb / 3.0;
    }
    for (int j = 0; j < 3; ++j) s -= 2.0 * P->Atu[i][j] * P->dal[j];
    double t = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) t += P->Gu[i][j][k] * P->Atu[j][k];
    for (int j = 0; j < 3; ++j) t += 6.0 * P->Atu[i][j] * P->dphi[j];
    for (int j = 0; j < 3; ++j) t -= (2.0 / 3.0) * gtu[i][j] * P->dK[j];
    s += 2.0 * al * t;
    rXt[i] = s;
    out[14 + i] = s;
  }
  /* lapse */
  if (prm->slicing == 0)
    out[17] = adv[17] - 2.0 * al * K;
  else if (prm->slicing == 1)
    out[17] = adv[17] - al * al * K;
  else
    out[17] = 0.0;
  /* shift and B */
  for (int i = 0; i < 3; ++i) {
    if (prm->shift == 0) {
      out[18 + i] = adv[18 + i] + 0.75 * u[21 + i];
      out[21 + i] = adv[21 + i] + (rXt[i] - adv[14 + i]) - prm->eta * u[21 + i];
    } else {
      out[18 + i] = 0.0;
      out[21 + i] = 0.0;
    }
  }
}

static int frozen_var_(int v, const orc_params* prm) {
  if (v == 17 && prm->slicing == 2) return 1;
  if (v >= 18 && prm->shift == 1) return 1;
  return 0;
}

/* BSSN right-hand side including Kreiss-Oliger dissipation on every evolved
 * (non-frozen) variable.  Ghosts of st must be valid. */
void orc_bssn_rhs(const double* st, double* rhs, const orc_grid* G, const orc_params* prm) {
  const size_t fs = fsize_(G);
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const double ko_scale = prm->eps_diss / (64.0 * G->h);
  const int g = G->g;
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = g; k < g + G->nz; ++k) {
    bssn_pt* P = (bssn_pt*)malloc(sizeof(bssn_pt));
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        memset(P, 0, sizeof(*P));
        bssn_load_(st, fs, str, c, G->h, P);
        double out[24];
        bssn_point_rhs_(P, prm, out);
        for (int v = 0; v < 24; ++v) {
          double r = out[v];
          if (!frozen_var_(v, prm)) {
            const double* p = st + (size_t)v * fs + c;
            double ko = st_ko(p, str[0]) + st_ko(p, str[1]) + st_ko(p, str[2]);
            r += ko_scale * ko;
          }
          rhs[(size_t)v * fs + c] = r;
        }
      }
    free(P);
  }
}

/* BSSN constraints on the interior: out has 7 grid functions
 *   0: Hamiltonian H = R + 2/3 K^2 - At_ij At^ij,  R = e^{-4phi} gt^ij R_ij
 *   1-3: momentum M^i = d_j At^ij + Gamma~^i_jk At^jk + 6 At^ij d_j phi
 *                       - 2/3 gt^ij d_j K   (d_j At^ij by the product rule)
 *   4-6: Gamma-constraint G^i = Xt^i - Gamma~^i_(d). */
void orc_bssn_constraints(const double* st, double* out, const orc_grid* G) {
  const size_t fs = fsize_(G);
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const int g = G->g;
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = g; k < g + G->nz; ++k) {
    bssn_pt* P = (bssn_pt*)malloc(sizeof(bssn_pt));
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        memset(P, 0, sizeof(*P));
        bssn_load_(st, fs, str, c, G->h, P);
        double R[3][3], DDal[3][3], trDDal;
        bssn_ricci_(P, R, DDal, &trDDal);
        const double (*gtu)[3] = (const double (*)[3])P->gtu;
        double trR = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) trR += gtu[a][b] * R[a][b];
        double K = P->u[7];
        out[c] = P->e4 * trR + (2.0 / 3.0) * K * K - P->AA;
        /* derivative of the inverse metric: dgtu[i][j][k] = d_k gt^ij */
        double dgtu[3][3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            for (int kk = 0; kk < 3; ++kk) {
              double s = 0.0;
              for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) s += gtu[a][p] * gtu[b][q] * P->dgt[p][q][kk];
              dgtu[a][b][kk] = -s;
            }
        for (int a = 0; a < 3; ++a) {
          double div = 0.0;
          for (int jj = 0; jj < 3; ++jj)
            for (int p = 0; p < 3; ++p)
              for (int q = 0; q < 3; ++q)
                div += dgtu[a][p][jj] * gtu[jj][q] * P->At[p][q] +
                       gtu[a][p] * dgtu[jj][q][jj] * P->At[p][q] +
                       gtu[a][p] * gtu[jj][q] * P->dAt[p][q][jj];
          double s = div;
          for (int jj = 0; jj < 3; ++jj)
            for (int kk = 0; kk < 3; ++kk) s += P->Gu[a][jj][kk] * P->Atu[jj][kk];
          for (int jj = 0; jj < 3; ++jj) s += 6.0 * P->Atu[a][jj] * P->dphi[jj];
          for (int jj = 0; jj < 3; ++jj) s -= (2.0 / 3.0) * gtu[a][jj] * P->dK[jj];
          out[(size_t)(1 + a) * fs + c] = s;
          out[(size_t)(4 + a) * fs + c] = P->u[14 + a] - P->Xtn[a];
        }
      }
    free(P);
  }
}

/* ------------------------------------------------------------------ */
/* Method of lines: classic RK4 (Sec. 2, time integrator).             */
/* ------------------------------------------------------------------ */
static int nvars_of_(int kind) { return kind == ORC_BSSN ? 24 : (kind == ORC_WAVE1 ? 5 : 2); }

int orc_rhs(int kind, const double* st, const double* s, double* rhs, const orc_grid* G,
            const orc_params* prm) {
  const int order = (prm && prm->order) ? prm->order : 4;
  switch (kind) {
    case ORC_WAVE:
      if (order != 4) return orc_wave_rhs_order(st, rhs, G, order);
      orc_wave_rhs(st, rhs, G);
      return 0;
    case ORC_WAVE1: return orc_wave1_rhs(st, rhs, G, order);
    case ORC_WAVE_VARC: orc_varc_rhs(st, s, rhs, G); return 0;
    case ORC_BSSN: orc_bssn_rhs(st, rhs, G, prm); return 0;
    default: return -1;
  }
}

/* y_out = y + a*k on the interior of nv grid functions */
static void axpy_int_(double* yo, const double* y, double a, const double* kk, int nv,
                      const orc_grid* G) {
  const size_t fs = fsize_(G);
  const int g = G->g;
  for (int v = 0; v < nv; ++v) {
#pragma omp parallel for schedule(static)
    for (int k = g; k < g + G->nz; ++k)
      for (int j = g; j < g + G->ny; ++j)
        for (int i = g; i < g + G->nx; ++i) {
          size_t c = (size_t)v * fs + (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
          yo[c] = y[c] + a * kk[c];
        }
  }
}

/* One classic RK4 step y <- y + dt/6 (k1 + 2k2 + 2k3 + k4); the ghosts of y
 * are refilled before each stage and on return.  work holds 5 states. */
static void rk4_one_(int kind, double* y, const double* s, const orc_grid* G,
                     const orc_params* prm, double dt, double* work) {
  const int nv = nvars_of_(kind);
  const size_t n = (size_t)nv * fsize_(G);
  double *k1 = work, *k2 = work + n, *k3 = work + 2 * n, *k4 = work + 3 * n, *yt = work + 4 * n;
  const size_t fs = fsize_(G);
  const int g = G->g;
  memcpy(yt, y, n * sizeof(double));
  orc_fill_ghosts(y, nv, G);
  orc_rhs(kind, y, s, k1, G, prm);
  axpy_int_(yt, y, 0.5 * dt, k1, nv, G);
  orc_fill_ghosts(yt, nv, G);
  orc_rhs(kind, yt, s, k2, G, prm);
  axpy_int_(yt, y, 0.5 * dt, k2, nv, G);
  orc_fill_ghosts(yt, nv, G);
  orc_rhs(kind, yt, s, k3, G, prm);
  axpy_int_(yt, y, dt, k3, nv, G);
  orc_fill_ghosts(yt, nv, G);
  orc_rhs(kind, yt, s, k4, G, prm);
  for (int v = 0; v < nv; ++v) {
#pragma omp parallel for schedule(static)
    for (int k = g; k < g + G->nz; ++k)
      for (int j = g; j < g + G->ny; ++j)
        for (int i = g; i < g + G->nx; ++i) {
          size_t c = (size_t)v * fs + (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
          y[c] = y[c] + (dt / 6.0) * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
        }
  }
  orc_fill_ghosts(y, nv, G);
}

int orc_rk4(int kind, double* y, const double* s, const orc_grid* G, const orc_params* prm,
            double dt, int nsteps) {
  const int nv = nvars_of_(kind);
  double* work = (double*)calloc((size_t)5 * nv * fsize_(G), sizeof(double));
  if (!work) return -2;
  for (int n = 0; n < nsteps; ++n) rk4_one_(kind, y, s, G, prm, dt, work);
  if (nsteps == 0) orc_fill_ghosts(y, nv, G);
  free(work);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Differentiation of the variable-speed wave RK4 map.                 */
/* ------------------------------------------------------------------ */

/* Tangent-linear RK4: advances the state y and, alongside it, the tangent dy
 * in the direction (dy, ds) of the initial state and of s = c^2.  Ghosts of
 * s and ds must be valid. */
int orc_varc_tlm_rk4(double* y, double* dy, const double* s, const double* ds,
                     const orc_grid* G, double dt, int nsteps) {
  const size_t n = 2 * fsize_(G);
  double* w = (double*)calloc(10 * n, sizeof(double));
  if (!w) return -2;
  double *yt = w, *dyt = w + n, *k[4], *dk[4];
  for (int q = 0; q < 4; ++q) { k[q] = w + (2 + q) * n; dk[q] = w + (6 + q) * n; }
  const double c[4] = {0.0, 0.5, 0.5, 1.0};
  const double b[4] = {1.0, 2.0, 2.0, 1.0};
  orc_params none = {0, 0, 0, 0, 0};
  for (int step = 0; step < nsteps; ++step) {
    orc_fill_ghosts(y, 2, G);
    orc_fill_ghosts(dy, 2, G);
    for (int q = 0; q < 4; ++q) {
      if (q == 0) {
        memcpy(yt, y, n * sizeof(double));
        memcpy(dyt, dy, n * sizeof(double));
      } else {
        axpy_int_(yt, y, c[q] * dt, k[q - 1], 2, G);
        axpy_int_(dyt, dy, c[q] * dt, dk[q - 1], 2, G);
        orc_fill_ghosts(yt, 2, G);
        orc_fill_ghosts(dyt, 2, G);
      }
      orc_rhs(ORC_WAVE_VARC, yt, s, k[q], G, &none);
      orc_varc_tlm_rhs(yt, s, dyt, ds, dk[q], G);
    }
    const size_t fs = fsize_(G);
    const int g = G->g;
    for (int v = 0; v < 2; ++v) {
#pragma omp parallel for schedule(static)
      for (int kk = g; kk < g + G->nz; ++kk)
        for (int j = g; j < g + G->ny; ++j)
          for (int i = g; i < g + G->nx; ++i) {
            size_t p = (size_t)v * fs + (size_t)kk * plane_(G) + (size_t)j * px_(G) + i;
            y[p] = y[p] + (dt / 6.0) * (b[0] * k[0][p] + b[1] * k[1][p] + b[2] * k[2][p] + b[3] * k[3][p]);
            dy[p] = dy[p] + (dt / 6.0) * (b[0] * dk[0][p] + b[1] * dk[1][p] + b[2] * dk[2][p] + b[3] * dk[3][p]);
          }
    }
  }
  orc_fill_ghosts(y, 2, G);
  orc_fill_ghosts(dy, 2, G);
  free(w);
  return 0;
}

/* Stage-wise reverse of one RK4 step taken from y_n (ghosts valid).  On entry
 * ybar holds the cotangent of y_{n+1}; on exit that of y_n.  sbar accumulates
 * the cotangent of s.  work holds 9 states of 2 variables. */
static void varc_rk4_reverse_one_(const double* yn, double* ybar, double* sbar, const double* s,
                                  const orc_grid* G, double dt, double* work) {
  const size_t n = 2 * fsize_(G);
  double* ys[4];
  double* ks[3];
  for (int q = 0; q < 4; ++q) ys[q] = work + q * n;
  for (int q = 0; q < 3; ++q) ks[q] = work + (4 + q) * n;
  double* kb = work + 7 * n; /* kbar of the current stage */
  double* kbq[4];            /* kbar_1..kbar_4 */
  double* yhat = work + 8 * n;
  orc_params none = {0, 0, 0, 0, 0};
  /* recompute the stage states y1..y4 */
  memcpy(ys[0], yn, n * sizeof(double));
  orc_rhs(ORC_WAVE_VARC, ys[0], s, ks[0], G, &none);
  memcpy(ys[1], yn, n * sizeof(double));
  axpy_int_(ys[1], yn, 0.5 * dt, ks[0], 2, G);
  orc_fill_ghosts(ys[1], 2, G);
  orc_rhs(ORC_WAVE_VARC, ys[1], s, ks[1], G, &none);
  memcpy(ys[2], yn, n * sizeof(double));
  axpy_int_(ys[2], yn, 0.5 * dt, ks[1], 2, G);
  orc_fill_ghosts(ys[2], 2, G);
  orc_rhs(ORC_WAVE_VARC, ys[2], s, ks[2], G, &none);
  memcpy(ys[3], yn, n * sizeof(double));
  axpy_int_(ys[3], yn, dt, ks[2], 2, G);
  orc_fill_ghosts(ys[3], 2, G);
  /* the stage cotangents: kbar_q = b_q dt/6 ybar' (b = 1,2,2,1) */
  double* buf = (double*)calloc(4 * n, sizeof(double));
  for (int q = 0; q < 4; ++q) kbq[q] = buf + q * n;
  const double w[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
  for (int q = 0; q < 4; ++q)
    for (size_t p = 0; p < n; ++p) kbq[q][p] = w[q] * ybar[p];
  /* stage 4 back to stage 1: yhat = J^T kbar_q; ybar += yhat;
   * kbar_{q-1} += a_q dt yhat with a = (1/2, 1/2, 1) for q = 2, 3, 4. */
  const double a[4] = {0.0, 0.5, 0.5, 1.0};
  for (int q = 3; q >= 0; --q) {
    memcpy(kb, kbq[q], n * sizeof(double));
    memset(yhat, 0, n * sizeof(double));
    orc_varc_adj_rhs(ys[q], s, kb, yhat, sbar, G);
    for (size_t p = 0; p < n; ++p) ybar[p] += yhat[p];
    if (q > 0)
      for (size_t p = 0; p < n; ++p) kbq[q - 1][p] += a[q] * dt * yhat[p];
  }
  free(buf);
}

/* Vector-Jacobian product of the nsteps-step RK4 map of the variable-speed
 * wave equation: given the cotangent ybar of the final state (2 grid
 * functions, interior), returns in ybar the cotangent of the initial state y0
 * and adds to sbar the cotangent of s.  Checkpoints of y_n are kept every
 * ckpt_every steps and the steps of each segment recomputed from its
 * checkpoint, newest segment first.  s must have valid ghosts. */
int orc_varc_vjp(const double* y0, const double* s, const orc_grid* G, double dt, int nsteps,
                 int ckpt_every, double* ybar, double* sbar) {
  if (ckpt_every <= 0 || nsteps < 0) return -1;
  const size_t fs = fsize_(G), n = 2 * fs;
  const int nck = nsteps == 0 ? 1 : (nsteps + ckpt_every - 1) / ckpt_every;
  double* ck = (double*)calloc((size_t)nck * n, sizeof(double));
  double* y = (double*)calloc(n, sizeof(double));
  double* work = (double*)calloc(10 * n, sizeof(double));
  double* seg = (double*)calloc((size_t)ckpt_every * n, sizeof(double));
  if (!ck || !y || !work || !seg) { free(ck); free(y); free(work); free(seg); return -2; }
  orc_params none = {0, 0, 0, 0, 0};
  memcpy(y, y0, n * sizeof(double));
  orc_fill_ghosts(y, 2, G);
  for (int st = 0; st < nsteps; ++st) {
    if (st % ckpt_every == 0) memcpy(ck + (size_t)(st / ckpt_every) * n, y, n * sizeof(double));
    rk4_one_(ORC_WAVE_VARC, y, s, G, &none, dt, work);
  }
  for (int sg = nck - 1; sg >= 0 && nsteps > 0; --sg) {
    int n0 = sg * ckpt_every, n1 = n0 + ckpt_every;
    if (n1 > nsteps) n1 = nsteps;
    memcpy(seg, ck + (size_t)sg * n, n * sizeof(double));
    for (int st = n0 + 1; st < n1; ++st) {
      double* dst = seg + (size_t)(st - n0) * n;
      memcpy(dst, seg + (size_t)(st - n0 - 1) * n, n * sizeof(double));
      rk4_one_(ORC_WAVE_VARC, dst, s, G, &none, dt, work);
    }
    for (int st = n1 - 1; st >= n0; --st)
      varc_rk4_reverse_one_(seg + (size_t)(st - n0) * n, ybar, sbar, s, G, dt, work);
  }
  free(ck); free(y); free(work); free(seg);
  return 0;
}

static void zero_ghosts_(double* a, const orc_grid* G) {
  const int g = G->g;
  for (int k = 0; k < (int)pz_(G); ++k)
    for (int j = 0; j < (int)py_(G); ++j)
      for (int i = 0; i < (int)px_(G); ++i) {
        int interior = i >= g && i < g + G->nx && j >= g && j < g + G->ny && k >= g && k < g + G->nz;
        if (!interior) a[(size_t)k * plane_(G) + (size_t)j * px_(G) + i] = 0.0;
      }
}

/* Gradient of J = 1/2 sum_r (u_N(x_r) - d_r)^2 after nsteps RK4 steps of the
 * variable-speed wave equation, with respect to the initial state and s.
 * recv holds padded linear indices into one grid function (interior
 * points).  The seed of the reverse sweep is ubar_N(x_r) = u_N(x_r) - d_r.
 * grad_y0 (2 grid functions) and grad_s are written on the interior; their
 * ghosts are zero. */
int orc_varc_adjoint(const double* y0, const double* s, const orc_grid* G, double dt, int nsteps,
                     int ckpt_every, const int64_t* recv, int nrecv, const double* data,
                     double* loss, double* grad_y0, double* grad_s) {
  if (ckpt_every <= 0 || nsteps < 0) return -1;
  const size_t fs = fsize_(G), n = 2 * fs;
  double* y = (double*)calloc(n, sizeof(double));
  if (!y) return -2;
  orc_params none = {0, 0, 0, 0, 0};
  memcpy(y, y0, n * sizeof(double));
  int rc = orc_rk4(ORC_WAVE_VARC, y, s, G, &none, dt, nsteps);
  if (rc) { free(y); return rc; }
  double J = 0.0;
  memset(grad_y0, 0, n * sizeof(double));
  memset(grad_s, 0, fs * sizeof(double));
  for (int r = 0; r < nrecv; ++r) {
    double m = y[recv[r]] - data[r];
    J += 0.5 * m * m;
    grad_y0[recv[r]] += m;
  }
  *loss = J;
  free(y);
  rc = orc_varc_vjp(y0, s, G, dt, nsteps, ckpt_every, grad_y0, grad_s);
  zero_ghosts_(grad_y0, G);
  zero_ghosts_(grad_y0 + fs, G);
  zero_ghosts_(grad_s, G);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Finite differencing of arbitrary (even) order (Sec. 3.2.2: "standard" */
/* operators of arbitrary order).  Central weights for order p = 2m:    */
/*   D1 f = (1/h)   sum_k a_k (f_k - f_-k),                            */
/*   a_k  = (-1)^(k+1) (m!)^2 / (k (m-k)! (m+k)!)                      */
/*   D2 f = (1/h^2) sum_k b_k ((f_k - f_0) + (f_-k - f_0)),            */
/*   b_k  = 2 (-1)^(k+1) (m!)^2 / (k^2 (m-k)! (m+k)!)                  */
/* ------------------------------------------------------------------ */
static double fact_(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

int orc_fd_weights(int order, double* a, double* b) {
  if (order < 2 || order > 16 || order % 2) return -1;
  const int m = order / 2;
  for (int k = 1; k <= m; ++k) {
    const double sgn = (k % 2) ? 1.0 : -1.0;
    const double c = fact_(m) * fact_(m) / (fact_(m - k) * fact_(m + k));
    a[k - 1] = sgn * c / k;
    b[k - 1] = 2.0 * sgn * c / ((double)k * k);
  }
  return 0;
}

static double st_d1o_(const double* p, ptrdiff_t s, int m, const double* a) {
  double r = 0.0;
  for (int k = m; k >= 1; --k) r += a[k - 1] * (p[k * s] - p[-k * s]);
  return r;
}

static double st_d2o_(const double* p, ptrdiff_t s, int m, const double* b) {
  const double f0 = p[0];
  double r = 0.0;
  for (int k = m; k >= 1; --k) r += b[k - 1] * ((p[k * s] - f0) + (p[-k * s] - f0));
  return r;
}

/* Order-p derivative field on the interior: kind 0 D1, kind 1 D2 along a. */
int orc_deriv_order(const double* f, double* out, const orc_grid* G, int order, int kind, int a) {
  double wa[8], wb[8];
  if (orc_fd_weights(order, wa, wb) || G->g < order / 2) return -1;
  const int m = order / 2;
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const double ih = 1.0 / G->h, ih2 = 1.0 / (G->h * G->h);
  const int g = G->g;
#pragma omp parallel for schedule(static)
  for (int k = g; k < g + G->nz; ++k)
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        out[c] = kind == 0 ? st_d1o_(f + c, str[a], m, wa) * ih : st_d2o_(f + c, str[a], m, wb) * ih2;
      }
  return 0;
}

/* Scalar wave, two-variable form, order-p Laplacian. */
int orc_wave_rhs_order(const double* st, double* rhs, const orc_grid* G, int order) {
  double wa[8], wb[8];
  if (orc_fd_weights(order, wa, wb) || G->g < order / 2) return -1;
  const int m = order / 2;
  const size_t fs = fsize_(G);
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const double ih2 = 1.0 / (G->h * G->h);
  const int g = G->g;
#pragma omp parallel for schedule(static)
  for (int k = g; k < g + G->nz; ++k)
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        double lap = 0.0;
        for (int d = 0; d < 3; ++d) lap += st_d2o_(st + c, str[d], m, wb) * ih2;
        rhs[c] = st[fs + c];
        rhs[fs + c] = lap;
      }
  return 0;
}

/* Scalar wave in the first-order form of Eq. 1 (5 variables u, rho, v_x,
 * v_y, v_z): u_t = rho, rho_t = sum_i D_i v_i, (v_i)_t = D_i rho, with
 * order-p first derivatives. */
int orc_wave1_rhs(const double* st, double* rhs, const orc_grid* G, int order) {
  double wa[8], wb[8];
  if (orc_fd_weights(order, wa, wb) || G->g < order / 2) return -1;
  const int m = order / 2;
  const size_t fs = fsize_(G);
  const ptrdiff_t str[3] = {1, (ptrdiff_t)px_(G), (ptrdiff_t)plane_(G)};
  const double ih = 1.0 / G->h;
  const int g = G->g;
#pragma omp parallel for schedule(static)
  for (int k = g; k < g + G->nz; ++k)
    for (int j = g; j < g + G->ny; ++j)
      for (int i = g; i < g + G->nx; ++i) {
        size_t c = (size_t)k * plane_(G) + (size_t)j * px_(G) + i;
        double div = 0.0;
        for (int d = 0; d < 3; ++d) div += st_d1o_(st + (size_t)(2 + d) * fs + c, str[d], m, wa) * ih;
        rhs[c] = st[fs + c];
        rhs[fs + c] = div;
        for (int d = 0; d < 3; ++d) rhs[(size_t)(2 + d) * fs + c] = st_d1o_(st + fs + c, str[d], m, wa) * ih;
      }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Two-level mesh refinement with Berger-Oliger subcycling (Sec. 4: the */
/* Carpet driver's AMR with subcycling in time), 4th-order systems.     */
/*                                                                      */
/* Coarse level: periodic grid of spacing H.  Fine level: nbox boxes;   */
/* box b refines the coarse points [lo_b, hi_b) per axis by 2 (spacing  */
/* H/2); its interior holds the fine points of global fine index        */
/* 2 lo_b .. 2 hi_b - 1 and its ghost zones (width g_f, the buffer) are */
/* filled by prolongation from the coarse level only: quintic Lagrange  */
/* interpolation along each axis (weights 3, -25, 150, 150, -25, 3 over */
/* 256 at fine points between coarse points, injection at coincident    */
/* ones) of a linear combination of coarse time levels (the time        */
/* interpolation).  Restriction: injection of the fine values at        */
/* coincident points into the coarse interior.  Boxes do not overlap.   */
/* ------------------------------------------------------------------ */
typedef struct {
  int nc[3], gc; /* coarse points along x, y, z; coarse ghosts */
  int nbox;      /* fine boxes */
  const int* lo; /* 3 * nbox: box b covers coarse points [lo[3b+d], hi[3b+d]) along axis d */
  const int* hi;
  int gf;        /* fine ghosts: the buffer width */
  double H;      /* coarse spacing */
} orc_amrn;

/* the single-box, scalar-wave configuration of the first interface */
typedef struct {
  int nc, gc;
  int lo[3], hi[3];
  int gf;
  double H;
} orc_amr;

static int amrn_nf_(const orc_amrn* A, int b, int d) { return 2 * (A->hi[3 * b + d] - A->lo[3 * b + d]); }

static orc_grid amrn_fine_grid_(const orc_amrn* A, int b) {
  orc_grid G = {amrn_nf_(A, b, 0), amrn_nf_(A, b, 1), amrn_nf_(A, b, 2), A->gf, 0.5 * A->H};
  return G;
}

/* 0 if every box lies where its prolongation reads valid coarse points:
 * box b reads the coarse points [lo - g_f/2 - 2, hi + g_f/2 + 2] per axis
 * (the buffer's g_f/2 coarse points and the quintic's reach), which must be
 * inside the padded coarse grid; g_f even; boxes pairwise disjoint. */
static int amrn_check_(const orc_amrn* A) {
  if (A->nbox < 1 || A->gf < 2 || A->gf % 2 || A->gc < 0) return -1;
  for (int b = 0; b < A->nbox; ++b)
    for (int d = 0; d < 3; ++d) {
      const int lo = A->lo[3 * b + d], hi = A->hi[3 * b + d];
      if (hi <= lo || lo - A->gf / 2 - 2 < -A->gc || hi + A->gf / 2 + 2 > A->nc[d] + A->gc - 1) return -1;
    }
  for (int a = 0; a < A->nbox; ++a)
    for (int b = a + 1; b < A->nbox; ++b) {
      int overlap = 1;
      for (int d = 0; d < 3; ++d)
        if (A->hi[3 * a + d] <= A->lo[3 * b + d] || A->hi[3 * b + d] <= A->lo[3 * a + d]) overlap = 0;
      if (overlap) return -1;
    }
  return 0;
}

/* weights of coarse points (global coarse index) for fine global index F */
static int prolong_w_(int F, int* base, double* w) {
  if (F % 2 == 0) {
    *base = F / 2;
    w[0] = 1.0;
    return 1;
  }
  const int I = (F - 1) / 2;  /* F = 2 I + 1 (exact: F - 1 is even) */
  *base = I - 2;
  w[0] = 3.0 / 256.0;
  w[1] = -25.0 / 256.0;
  w[2] = 150.0 / 256.0;
  w[3] = 150.0 / 256.0;
  w[4] = -25.0 / 256.0;
  w[5] = 3.0 / 256.0;
  return 6;
}

/* Fill the ghost zones of nv grid functions `fine` of box b from coarse
 * levels c[0..nt-1] (each nv grid functions, periodic ghosts valid) with
 * time weights tw[0..nt-1]. */
int orc_amrn_prolong(const orc_amrn* A, int b, int nv, const double* const* c, const double* tw, int nt,
                     double* fine) {
  if (amrn_check_(A) || b < 0 || b >= A->nbox) return -1;
  orc_grid Gc = {A->nc[0], A->nc[1], A->nc[2], A->gc, A->H};
  orc_grid Gf = amrn_fine_grid_(A, b);
  const int* lo = A->lo + 3 * b;
  const size_t fsc = fsize_(&Gc), fsf = fsize_(&Gf);
  const int pfx = (int)px_(&Gf), pfy = (int)py_(&Gf), pfz = (int)pz_(&Gf);
  const int nf[3] = {Gf.nx, Gf.ny, Gf.nz};
  for (int v = 0; v < nv; ++v)
#pragma omp parallel for schedule(static)
    for (int k = 0; k < pfz; ++k)
      for (int j = 0; j < pfy; ++j)
        for (int i = 0; i < pfx; ++i) {
          const int P[3] = {i, j, k};
          int interior = 1;
          for (int d = 0; d < 3; ++d)
            if (P[d] < A->gf || P[d] >= A->gf + nf[d]) interior = 0;
          if (interior) continue;
          int base[3], n[3];
          double w[3][6];
          for (int d = 0; d < 3; ++d) {
            const int F = 2 * lo[d] + (P[d] - A->gf);
            n[d] = prolong_w_(F, &base[d], w[d]);
          }
          double val = 0.0;
          for (int t = 0; t < nt; ++t) {
            const double* cv = c[t] + (size_t)v * fsc;
            double s = 0.0;
            for (int c2 = 0; c2 < n[2]; ++c2)
              for (int c1 = 0; c1 < n[1]; ++c1)
                for (int c0 = 0; c0 < n[0]; ++c0) {
                  const size_t q = (size_t)(base[2] + c2 + A->gc) * plane_(&Gc) +
                                   (size_t)(base[1] + c1 + A->gc) * px_(&Gc) + (base[0] + c0 + A->gc);
                  s += w[2][c2] * w[1][c1] * w[0][c0] * cv[q];
                }
            val += tw[t] * s;
          }
          fine[(size_t)v * fsf + (size_t)k * plane_(&Gf) + (size_t)j * px_(&Gf) + i] = val;
        }
  return 0;
}

/* Coarse interior points of box b take the coincident fine values. */
int orc_amrn_restrict(const orc_amrn* A, int b, int nv, const double* fine, double* coarse) {
  if (b < 0 || b >= A->nbox || A->gf < 0) return -1;
  for (int d = 0; d < 3; ++d)  /* the box's coarse points lie in the coarse interior */
    if (A->lo[3 * b + d] < 0 || A->hi[3 * b + d] > A->nc[d] || A->hi[3 * b + d] <= A->lo[3 * b + d]) return -1;
  orc_grid Gc = {A->nc[0], A->nc[1], A->nc[2], A->gc, A->H};
  orc_grid Gf = amrn_fine_grid_(A, b);
  const int* lo = A->lo + 3 * b;
  const int* hi = A->hi + 3 * b;
  const size_t fsc = fsize_(&Gc), fsf = fsize_(&Gf);
  for (int v = 0; v < nv; ++v)
    for (int K = lo[2]; K < hi[2]; ++K)
      for (int J = lo[1]; J < hi[1]; ++J)
        for (int I = lo[0]; I < hi[0]; ++I) {
          const size_t qc = (size_t)(K + A->gc) * plane_(&Gc) + (size_t)(J + A->gc) * px_(&Gc) + (I + A->gc);
          const size_t qf = (size_t)(2 * (K - lo[2]) + A->gf) * plane_(&Gf) +
                            (size_t)(2 * (J - lo[1]) + A->gf) * px_(&Gf) + (2 * (I - lo[0]) + A->gf);
          coarse[(size_t)v * fsc + qc] = fine[(size_t)v * fsf + qf];
        }
  return 0;
}

/* stencil radius of a system's right-hand side (4th order; BSSN: the
 * 7-point dissipation stencil) */
static int amrn_radius_(int kind) { return kind == ORC_BSSN ? 3 : 2; }

/* nsteps Berger-Oliger steps of the two-level system `kind` (ORC_WAVE or
 * ORC_BSSN with parameters prm), coarse step dt.  Each fine box's ghost
 * zone of width g_f >= 4 r (r the stencil radius: 2 for the wave, 3 for
 * BSSN) is a buffer: it is filled by prolongation at the start of each fine
 * step, and the four RK stages are evaluated on the box interior extended
 * by g_f - r points, a region whose valid part shrinks by r per stage, so
 * the interior stays valid.  Coarse data at the fine step's start time
 * t_n + theta dt come from cubic Hermite interpolation through (y_n, k_n)
 * and (y_{n+1}, k_{n+1}), k the coarse right-hand side.  Per coarse step:
 *   1. k_n = RHS(y_n); one coarse RK4 step to y_{n+1}; k_{n+1} = RHS(y_{n+1});
 *   2. for every box, two fine RK4 steps of dt/2, the buffer prolonged at
 *      theta = 0, 1/2;
 *   3. restrict every box into the coarse interior and refill the coarse
 *      periodic ghosts.
 * coarse: padded state (ghosts g_c); fines[b]: padded state of box b
 * (ghosts g_f).  Returns -1 for an invalid configuration (amrn_check_),
 * -2 when out of memory. */
int orc_amrn_step(const orc_amrn* A, int kind, const orc_params* prm, double* coarse, double* const* fines,
                  double dt, int nsteps) {
  if (kind != ORC_WAVE && kind != ORC_BSSN) return -1;
  const int r = amrn_radius_(kind);
  if (amrn_check_(A) || A->gf < 4 * r || A->gc < r) return -1;
  const int nv = nvars_of_(kind);
  orc_grid Gc = {A->nc[0], A->nc[1], A->nc[2], A->gc, A->H};
  const size_t ncv = (size_t)nv * fsize_(&Gc);
  size_t nfmax = 0;
  for (int b = 0; b < A->nbox; ++b) {
    orc_grid Gf = amrn_fine_grid_(A, b);
    if ((size_t)nv * fsize_(&Gf) > nfmax) nfmax = (size_t)nv * fsize_(&Gf);
  }
  double* yn = (double*)malloc(ncv * sizeof(double));
  double* kn = (double*)calloc(ncv, sizeof(double));
  double* kn1 = (double*)calloc(ncv, sizeof(double));
  double* work = (double*)calloc(5 * nfmax, sizeof(double));
  double* cwork = (double*)calloc(5 * ncv, sizeof(double));
  if (!yn || !kn || !kn1 || !work || !cwork) {
    free(yn); free(kn); free(kn1); free(work); free(cwork);
    return -2;
  }
  const double dtf = 0.5 * dt;
  const double cst[4] = {0.0, 0.5, 0.5, 1.0};
  for (int n = 0; n < nsteps; ++n) {
    orc_fill_ghosts(coarse, nv, &Gc);
    memcpy(yn, coarse, ncv * sizeof(double));
    orc_rhs(kind, yn, NULL, kn, &Gc, prm);
    orc_fill_ghosts(kn, nv, &Gc); /* the prolongation reads periodic images */
    rk4_one_(kind, coarse, NULL, &Gc, prm, dt, cwork);
    orc_rhs(kind, coarse, NULL, kn1, &Gc, prm);
    orc_fill_ghosts(kn1, nv, &Gc);
    const double* lv[4] = {yn, kn, coarse, kn1};
    for (int b = 0; b < A->nbox; ++b) {
      double* fine = fines[b];
      const int ext = A->gf - r;
      orc_grid Ge = {amrn_nf_(A, b, 0) + 2 * ext, amrn_nf_(A, b, 1) + 2 * ext, amrn_nf_(A, b, 2) + 2 * ext, r,
                     0.5 * A->H};
      const size_t nf = (size_t)nv * fsize_(&Ge);
      for (int m = 0; m < 2; ++m) {
        /* cubic Hermite weights at theta = m / 2 */
        const double th = 0.5 * m;
        const double tw[4] = {2 * th * th * th - 3 * th * th + 1, dt * (th * th * th - 2 * th * th + th),
                              -2 * th * th * th + 3 * th * th, dt * (th * th * th - th * th)};
        orc_amrn_prolong(A, b, nv, lv, tw, 4, fine);
        double *k1 = work, *k2 = work + nf, *k3 = work + 2 * nf, *k4 = work + 3 * nf, *yt = work + 4 * nf;
        double* ks[4] = {k1, k2, k3, k4};
        for (int st = 0; st < 4; ++st) {
          double* ys = st == 0 ? fine : yt;
          if (st > 0) {
            memcpy(yt, fine, nf * sizeof(double));
            axpy_int_(yt, fine, cst[st] * dtf, ks[st - 1], nv, &Ge);
          }
          orc_rhs(kind, ys, NULL, ks[st], &Ge, prm);
        }
        const size_t fs = fsize_(&Ge);
        const int g = Ge.g;
        for (int v = 0; v < nv; ++v)
          for (int kk = g; kk < g + Ge.nz; ++kk)
            for (int j = g; j < g + Ge.ny; ++j)
              for (int i = g; i < g + Ge.nx; ++i) {
                size_t c = (size_t)v * fs + (size_t)kk * plane_(&Ge) + (size_t)j * px_(&Ge) + i;
                fine[c] = fine[c] + (dtf / 6.0) * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
              }
      }
    }
    for (int b = 0; b < A->nbox; ++b) orc_amrn_restrict(A, b, nv, fines[b], coarse);
    orc_fill_ghosts(coarse, nv, &Gc);
  }
  free(yn); free(kn); free(kn1); free(work); free(cwork);
  return 0;
}

/* The single-box scalar-wave interface: the general routines with one box. */
static orc_amrn amr_one_(const orc_amr* A) {
  orc_amrn N = {{A->nc, A->nc, A->nc}, A->gc, 1, A->lo, A->hi, A->gf, A->H};
  return N;
}

int orc_amr_prolong(const orc_amr* A, int nv, const double* const* c, const double* tw, int nt,
                    double* fine) {
  orc_amrn N = amr_one_(A);
  return orc_amrn_prolong(&N, 0, nv, c, tw, nt, fine);
}

int orc_amr_restrict(const orc_amr* A, int nv, const double* fine, double* coarse) {
  orc_amrn N = amr_one_(A);
  return orc_amrn_restrict(&N, 0, nv, fine, coarse);
}

int orc_amr_step(const orc_amr* A, double* coarse, double* fine, double dt, int nsteps) {
  orc_amrn N = amr_one_(A);
  orc_params none = {0, 0, 0, 0, 0};
  double* fines[1] = {fine};
  return orc_amrn_step(&N, ORC_WAVE, &none, coarse, fines, dt, nsteps);
}
