/*
 * mg_oracle.c -- FP64 CPU oracle for "Learning optimal multigrid smoothers via
 * neural networks" (Huang, Li & Xi, arXiv 2102.12071).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow restatement of the method, written from
 * the paper, used to check the CUDA library.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it; it shares no code with the CUDA
 * path.  Everything is double precision and follows the paper's steps in order,
 * with no blocking, fusion or reordering.  Conventions are in mg_oracle.h.
 *
 * Parity status of each part (what pins it) is listed in the test-suite; one part
 * is "parity unpinned": the paper's own trained network weights (never published),
 * which this oracle does not claim to reproduce.
 */
#include "mg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define KIDX(di, dj) (3 * ((di) + 1) + ((dj) + 1))

static int inside(int n, int i, int j) { return i >= 0 && i < n && j >= 0 && j < n; }

/* ------------------------------------------------------------------------- */
/* Discretisations                                                            */
/* ------------------------------------------------------------------------- */

/*
 * Bilinear (Q1) finite elements for -div(K grad u) = f (Sec. 3.1 eq. constant with a
 * tensor coefficient, Sec. 6.1 eq. pde), on the uniform mesh of the unit square with
 * (n+1) x (n+1) square cells and K constant on each cell.  The element matrix is
 * integrated exactly by 2x2 Gauss quadrature (the integrand is a polynomial of degree
 * 2 per variable); in 2-D it does not depend on the cell size h.  Cell (ci, cj),
 * 0 <= ci, cj <= n, spans mesh nodes ci..ci+1 (rows) and cj..cj+1 (columns); interior
 * unknown (i, j) is mesh node (i+1, j+1).  per_cell = 0: kxx, kxy, kyy point to one value.
 */
void or_fe_q1_field(int n, const double* kxx, const double* kxy, const double* kyy,
                    int per_cell, double* st) {
  const int nn = n * n;
  memset(st, 0, sizeof(double) * 9 * nn);
  const double g[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  /* gradients of the 4 bilinear shape functions at the 4 Gauss points;
     corner c = 2*yy + xx sits at (x, y) = (xx, yy). */
  double ke_unit[3][4][4]; /* [term xx / xy(sym) / yy][a][b] */
  memset(ke_unit, 0, sizeof(ke_unit));
  for (int qy = 0; qy < 2; ++qy)
    for (int qx = 0; qx < 2; ++qx) {
      const double x = g[qx], y = g[qy], w = 0.25;
      double gx[4], gy[4];
      for (int c = 0; c < 4; ++c) {
        const int xx = c & 1, yy = c >> 1;
        const double X = xx ? x : 1.0 - x, Y = yy ? y : 1.0 - y;
        gx[c] = (xx ? 1.0 : -1.0) * Y;
        gy[c] = (yy ? 1.0 : -1.0) * X;
      }
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          ke_unit[0][a][b] += w * gx[a] * gx[b];
          ke_unit[1][a][b] += w * (gx[a] * gy[b] + gy[a] * gx[b]);
          ke_unit[2][a][b] += w * gy[a] * gy[b];
        }
    }
  for (int ci = 0; ci <= n; ++ci)
    for (int cj = 0; cj <= n; ++cj) {
      const int cell = per_cell ? ci * (n + 1) + cj : 0;
      const double axx = kxx[cell], axy = kxy[cell], ayy = kyy[cell];
      for (int a = 0; a < 4; ++a) {
        const int pi = ci + (a >> 1) - 1, pj = cj + (a & 1) - 1; /* interior index of corner a */
        if (!inside(n, pi, pj)) continue;
        for (int b = 0; b < 4; ++b) {
          const int qi = ci + (b >> 1) - 1, qj = cj + (b & 1) - 1;
          if (!inside(n, qi, qj)) continue; /* Dirichlet node: not an unknown */
          const double v = axx * ke_unit[0][a][b] + axy * ke_unit[1][a][b] + ayy * ke_unit[2][a][b];
          st[KIDX(qi - pi, qj - pj) * nn + pi * n + pj] += v;
        }
      }
    }
}

/*
 * Interior Q1 stencil of the rotated anisotropic operator with
 * K = R(theta) diag(1, eps) R(theta)^T (Sec. 6.1 eq. pde with the conductivity
 * eps in place of xi; the tensor entries are those printed under eq. pde).
 */
void or_q1_rotated_stencil(double eps, double theta, double s[9]) {
  const double c = cos(theta), sn = sin(theta);
  const double kxx = c * c + eps * sn * sn;
  const double kxy = c * sn * (1.0 - eps);
  const double kyy = sn * sn + eps * c * c;
  double st[9 * 9];
  or_fe_q1_field(3, &kxx, &kxy, &kyy, 0, st); /* centre point of a 3x3 grid is interior */
  for (int k = 0; k < 9; ++k) s[k] = st[k * 9 + 4];
}

/*
 * Finite-difference form used for the spectral radii of Sec. 6.1 (Table 1):
 * A u = -(T11 u_xx + 2 T12 u_xy + T22 u_yy) with three-point second differences and
 * the seven-point u_xy stencil printed under eq. pde, T as printed there, h = 1
 * (a common scale factor does not change any spectral radius).
 */
void or_fd_rotated_stencil(double xi, double theta, double s[9]) {
  const double c = cos(theta), sn = sin(theta);
  const double t11 = c * c + xi * sn * sn;
  const double t12 = c * sn * (1.0 - xi);
  const double t22 = sn * sn + xi * c * c;
  double uxx[9] = {0}, uyy[9] = {0}, uxy[9] = {0};
  uxx[KIDX(0, -1)] = 1; uxx[KIDX(0, 0)] = -2; uxx[KIDX(0, 1)] = 1;
  uyy[KIDX(-1, 0)] = 1; uyy[KIDX(0, 0)] = -2; uyy[KIDX(1, 0)] = 1;
  /* rows of the printed stencil from top (north, di=+1) to bottom (south, di=-1) */
  uxy[KIDX(1, 0)] = -0.5; uxy[KIDX(1, 1)] = 0.5;
  uxy[KIDX(0, -1)] = -0.5; uxy[KIDX(0, 0)] = 1.0; uxy[KIDX(0, 1)] = -0.5;
  uxy[KIDX(-1, -1)] = 0.5; uxy[KIDX(-1, 0)] = -0.5;
  for (int k = 0; k < 9; ++k) s[k] = -(t11 * uxx[k] + 2.0 * t12 * uxy[k] + t22 * uyy[k]);
}

/* Variable-coefficient nine-point stencil printed in Sec. 4 (cell values g1..g4 around
   the point, h = 1): it is the Q1 element matrix with an isotropic cellwise coefficient. */
void or_paper9_field(int n, const double* g_cells, double* st) {
  const int nn = n * n;
  memset(st, 0, sizeof(double) * 9 * nn);
  const int nc = n + 1;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      /* cells around interior node (i, j): rows i (south) and i+1 (north),
         columns j (west) and j+1 (east). g1 = north-west, g2 = north-east,
         g3 = south-west, g4 = south-east (the printed u11 is the north-west corner). */
      const double g1 = g_cells[(i + 1) * nc + j], g2 = g_cells[(i + 1) * nc + j + 1];
      const double g3 = g_cells[i * nc + j], g4 = g_cells[i * nc + j + 1];
      double s[9];
      s[KIDX(1, -1)] = -g1 / 3.0;
      s[KIDX(1, 1)] = -g2 / 3.0;
      s[KIDX(-1, -1)] = -g3 / 3.0;
      s[KIDX(-1, 1)] = -g4 / 3.0;
      s[KIDX(1, 0)] = -(g1 + g2) / 6.0;
      s[KIDX(0, 1)] = -(g2 + g4) / 6.0;
      s[KIDX(-1, 0)] = -(g3 + g4) / 6.0;
      s[KIDX(0, -1)] = -(g1 + g3) / 6.0;
      s[KIDX(0, 0)] = 2.0 * (g1 + g2 + g3 + g4) / 3.0;
      for (int k = 0; k < 9; ++k) {
        const int di = k / 3 - 1, dj = k % 3 - 1;
        st[k * nn + i * n + j] = inside(n, i + di, j + dj) ? s[k] : 0.0;
      }
    }
}

/*
 * Five-point stencil of -div(a grad u) with a constant per cell and unknowns at the
 * mesh nodes: the flux across each mesh edge uses the mean of the two cells sharing
 * that edge (the five-point counterpart of the Sec. 4 nine-point formula), h = 1.
 */
void or_varcoef5_field(int n, const double* a, double* st) {
  const int nn = n * n, nc = n + 1;
  memset(st, 0, sizeof(double) * 9 * nn);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double wE = 0.5 * (a[i * nc + j + 1] + a[(i + 1) * nc + j + 1]);
      const double wW = 0.5 * (a[i * nc + j] + a[(i + 1) * nc + j]);
      const double wN = 0.5 * (a[(i + 1) * nc + j] + a[(i + 1) * nc + j + 1]);
      const double wS = 0.5 * (a[i * nc + j] + a[i * nc + j + 1]);
      const int p = i * n + j;
      st[KIDX(0, 0) * nn + p] = wE + wW + wN + wS;
      if (j + 1 < n) st[KIDX(0, 1) * nn + p] = -wE;
      if (j > 0) st[KIDX(0, -1) * nn + p] = -wW;
      if (i + 1 < n) st[KIDX(1, 0) * nn + p] = -wN;
      if (i > 0) st[KIDX(-1, 0) * nn + p] = -wS;
    }
}

/* The same constant stencil at every point, couplings across the boundary dropped. */
void or_const_field(int n, const double s[9], double* st) {
  const int nn = n * n;
  for (int k = 0; k < 9; ++k) {
    const int di = k / 3 - 1, dj = k % 3 - 1;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) st[k * nn + i * n + j] = inside(n, i + di, j + dj) ? s[k] : 0.0;
  }
}

/* ------------------------------------------------------------------------- */
/* Operators                                                                  */
/* ------------------------------------------------------------------------- */

/* y = A x (eq. Au=f) */
void or_apply(int n, const double* st, const double* x, double* y) {
  const int nn = n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 9; ++k) {
        const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
        if (inside(n, ii, jj)) acc += st[k * nn + i * n + j] * x[ii * n + jj];
      }
      y[i * n + j] = acc;
    }
}

/* Bilinear interpolation weight P(x, I) of fine point (fi, fj) from coarse point (I, J):
   full coarsening, coarse point I at fine 2I+1 (Sec. 6.1, Fig. full_coarsening). */
static double pweight(int fi, int fj, int ci, int cj) {
  const int dy = abs(fi - (2 * ci + 1)), dx = abs(fj - (2 * cj + 1));
  if (dy > 1 || dx > 1) return 0.0;
  return (1.0 - 0.5 * dy) * (1.0 - 0.5 * dx);
}

/* rc = P^T r: the restriction of Algorithm 1 (stencil 1/4 [1 2 1; 2 4 2; 1 2 1],
   four times the printed full weighting, so that P^T A P is the Galerkin operator). */
void or_restrict(int n, const double* r, double* rc) {
  const int nc = (n - 1) / 2;
  for (int I = 0; I < nc; ++I)
    for (int J = 0; J < nc; ++J) {
      double acc = 0.0;
      for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
          const int fi = 2 * I + 1 + di, fj = 2 * J + 1 + dj;
          acc += pweight(fi, fj, I, J) * r[fi * n + fj];
        }
      rc[I * nc + J] = acc;
    }
}

/* e += P ec (bilinear interpolation, Sec. 6.1). */
void or_prolong_add(int n, const double* ec, double* e) {
  const int nc = (n - 1) / 2;
  for (int I = 0; I < nc; ++I)
    for (int J = 0; J < nc; ++J)
      for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
          const int fi = 2 * I + 1 + di, fj = 2 * J + 1 + dj;
          e[fi * n + fj] += pweight(fi, fj, I, J) * ec[I * nc + J];
        }
}

/* Galerkin coarse operator P^T A P (Sec. 2.2), evaluated entry by entry:
   Ac(I, I+D) = sum_x sum_y P(x, I) A(x, y) P(y, I+D). */
void or_rap(int n, const double* st, double* stc) {
  const int nn = n * n, nc = (n - 1) / 2, nnc = nc * nc;
  for (int I = 0; I < nc; ++I)
    for (int J = 0; J < nc; ++J)
      for (int kc = 0; kc < 9; ++kc) {
        const int I2 = I + kc / 3 - 1, J2 = J + kc % 3 - 1;
        double acc = 0.0;
        if (inside(nc, I2, J2)) {
          for (int ai = -1; ai <= 1; ++ai)
            for (int aj = -1; aj <= 1; ++aj) {
              const int xi = 2 * I + 1 + ai, xj = 2 * J + 1 + aj;
              const double px = pweight(xi, xj, I, J);
              for (int k = 0; k < 9; ++k) {
                const int yi = xi + k / 3 - 1, yj = xj + k % 3 - 1;
                if (!inside(n, yi, yj)) continue;
                const double py = pweight(yi, yj, I2, J2);
                if (py == 0.0) continue;
                acc += px * st[k * nn + xi * n + xj] * py;
              }
            }
        }
        stc[kc * nnc + I * nc + J] = acc;
      }
}

/* Dense n^2 x n^2 matrix of a stencil field (row-major). */
void or_dense_matrix(int n, const double* st, double* A) {
  const int nn = n * n;
  memset(A, 0, sizeof(double) * (size_t)nn * nn);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < 9; ++k) {
        const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
        if (inside(n, ii, jj)) A[(size_t)(i * n + j) * nn + ii * n + jj] += st[k * nn + i * n + j];
      }
}

/* ------------------------------------------------------------------------- */
/* Smoothers                                                                  */
/* ------------------------------------------------------------------------- */

/* Weighted Jacobi M = omega^{-1} D (Sec. 2.1): H = omega D^{-1}, a 1-tap kernel. */
void or_jacobi_kernels(int n, const double* st, double omega, double* W) {
  const int nn = n * n;
  memset(W, 0, sizeof(double) * 9 * nn);
  for (int p = 0; p < nn; ++p) W[4 * nn + p] = omega / st[4 * nn + p];
}

/* y = H v with per-point (unshared) 3x3 kernels (Sec. 4). */
void or_apply_H(int n, const double* W, const double* v, double* y) {
  const int nn = n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 9; ++k) {
        const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
        if (inside(n, ii, jj)) acc += W[k * nn + i * n + j] * v[ii * n + jj];
      }
      y[i * n + j] = acc;
    }
}

/* y = H^T v: (H^T v)(q) = sum over p with q = p + d_k of W[k][p] v(p). */
void or_apply_HT(int n, const double* W, const double* v, double* y) {
  const int nn = n * n;
  memset(y, 0, sizeof(double) * nn);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < 9; ++k) {
        const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
        if (inside(n, ii, jj)) y[ii * n + jj] += W[k * nn + i * n + j] * v[i * n + j];
      }
}

/* u <- u + H (f - A u), nsteps times (eq. iteration with M^{-1} = H). */
void or_smooth(int n, const double* st, const double* W, const double* f, double* u, int nsteps) {
  const int nn = n * n;
  double* r = (double*)malloc(sizeof(double) * nn);
  double* hr = (double*)malloc(sizeof(double) * nn);
  for (int s = 0; s < nsteps; ++s) {
    or_apply(n, st, u, r);
    for (int p = 0; p < nn; ++p) r[p] = f[p] - r[p];
    or_apply_H(n, W, r, hr);
    for (int p = 0; p < nn; ++p) u[p] += hr[p];
  }
  free(r);
  free(hr);
}

/* One lexicographic Gauss-Seidel sweep, M = D - L (Sec. 2.1). */
void or_gauss_seidel(int n, const double* st, const double* f, double* u) {
  const int nn = n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = f[i * n + j];
      for (int k = 0; k < 9; ++k) {
        if (k == 4) continue;
        const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
        if (inside(n, ii, jj)) acc -= st[k * nn + i * n + j] * u[ii * n + jj];
      }
      u[i * n + j] = acc / st[4 * nn + i * n + j];
    }
}

/* ------------------------------------------------------------------------- */
/* Dense Cholesky (coarsest-level direct solve, Algorithm 1)                  */
/* ------------------------------------------------------------------------- */

int or_cholesky(int m, double* A) {
  for (int k = 0; k < m; ++k) {
    double d = A[(size_t)k * m + k];
    for (int t = 0; t < k; ++t) d -= A[(size_t)k * m + t] * A[(size_t)k * m + t];
    if (!(d > 0.0)) return -1;
    d = sqrt(d);
    A[(size_t)k * m + k] = d;
    for (int i = k + 1; i < m; ++i) {
      double v = A[(size_t)i * m + k];
      for (int t = 0; t < k; ++t) v -= A[(size_t)i * m + t] * A[(size_t)k * m + t];
      A[(size_t)i * m + k] = v / d;
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) A[(size_t)i * m + j] = 0.0;
  return 0;
}

void or_cholesky_solve(int m, const double* L, double* b) {
  for (int i = 0; i < m; ++i) {
    double v = b[i];
    for (int t = 0; t < i; ++t) v -= L[(size_t)i * m + t] * b[t];
    b[i] = v / L[(size_t)i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = b[i];
    for (int t = i + 1; t < m; ++t) v -= L[(size_t)t * m + i] * b[t];
    b[i] = v / L[(size_t)i * m + i];
  }
}

/* ------------------------------------------------------------------------- */
/* Hierarchy, V-cycle, solve (Algorithm 1; conventions of Sec. 3.1)           */
/* ------------------------------------------------------------------------- */

#define OR_MAXL 16
typedef struct {
  int L;                 /* number of levels; level L-1 is the coarsest */
  int n[OR_MAXL];
  double* st[OR_MAXL];   /* stencil fields: level 0 given, coarser = P^T A P */
  double* W[OR_MAXL];    /* smoothing kernels (levels 0..L-2) */
  double* chol;          /* dense Cholesky factor of the coarsest operator */
  int nu1, nu2;
} or_mg;

void* or_mg_create(int n, const double* st0, int coarsest_n, int nu1, int nu2) {
  or_mg* h = (or_mg*)calloc(1, sizeof(or_mg));
  h->nu1 = nu1;
  h->nu2 = nu2;
  int l = 0, m = n;
  h->n[0] = n;
  h->st[0] = (double*)malloc(sizeof(double) * 9 * n * n);
  memcpy(h->st[0], st0, sizeof(double) * 9 * n * n);
  while (m > coarsest_n && m >= 3 && (m - 1) % 2 == 0 && l + 1 < OR_MAXL) {
    const int mc = (m - 1) / 2;
    h->st[l + 1] = (double*)malloc(sizeof(double) * 9 * mc * mc);
    or_rap(m, h->st[l], h->st[l + 1]);
    h->n[l + 1] = mc;
    ++l;
    m = mc;
  }
  h->L = l + 1;
  for (int k = 0; k < h->L; ++k) {
    h->W[k] = (double*)malloc(sizeof(double) * 9 * h->n[k] * h->n[k]);
    or_jacobi_kernels(h->n[k], h->st[k], 2.0 / 3.0, h->W[k]);
  }
  const int mm = m * m;
  h->chol = (double*)malloc(sizeof(double) * (size_t)mm * mm);
  or_dense_matrix(m, h->st[h->L - 1], h->chol);
  if (or_cholesky(mm, h->chol) != 0) {
    or_mg_destroy(h);
    return NULL;
  }
  return h;
}

void or_mg_destroy(void* hv) {
  or_mg* h = (or_mg*)hv;
  if (!h) return;
  for (int k = 0; k < OR_MAXL; ++k) {
    free(h->st[k]);
    free(h->W[k]);
  }
  free(h->chol);
  free(h);
}

int or_mg_levels(void* h) { return ((or_mg*)h)->L; }
int or_mg_n(void* h, int level) { return ((or_mg*)h)->n[level]; }
void or_mg_get_field(void* hv, int l, double* st) {
  or_mg* h = (or_mg*)hv;
  memcpy(st, h->st[l], sizeof(double) * 9 * h->n[l] * h->n[l]);
}
void or_mg_get_kernels(void* hv, int l, double* W) {
  or_mg* h = (or_mg*)hv;
  memcpy(W, h->W[l], sizeof(double) * 9 * h->n[l] * h->n[l]);
}
void or_mg_set_kernels(void* hv, int l, const double* W) {
  or_mg* h = (or_mg*)hv;
  memcpy(h->W[l], W, sizeof(double) * 9 * h->n[l] * h->n[l]);
}
void or_mg_set_jacobi(void* hv, double omega) {
  or_mg* h = (or_mg*)hv;
  for (int k = 0; k < h->L; ++k) or_jacobi_kernels(h->n[k], h->st[k], omega, h->W[k]);
}
/* One network shared by every smoothed level; its input is each level's own stencil field. */
int or_mg_set_cnn(void* hv, const double* params, double omega, int bf16) {
  or_mg* h = (or_mg*)hv;
  for (int k = 0; k + 1 < h->L; ++k) or_hypernet_forward(h->n[k], h->st[k], params, omega, bf16, h->W[k]);
  return 0;
}

/* Algorithm 1 at level l on u (in place) with right-hand side f. */
static void vcycle_level(or_mg* h, int l, const double* f, double* u) {
  const int n = h->n[l], nn = n * n;
  or_smooth(n, h->st[l], h->W[l], f, u, h->nu1);             /* pre-smoothing */
  double* r = (double*)malloc(sizeof(double) * nn);
  or_apply(n, h->st[l], u, r);                                /* fine-level residual */
  for (int p = 0; p < nn; ++p) r[p] = f[p] - r[p];
  const int nc = h->n[l + 1], nnc = nc * nc;
  double* rc = (double*)malloc(sizeof(double) * nnc);
  double* uc = (double*)calloc(nnc, sizeof(double));
  or_restrict(n, r, rc);                                      /* r^(l+1) = P^T r^(l) */
  if (l + 1 == h->L - 1) {
    memcpy(uc, rc, sizeof(double) * nnc);                     /* coarsest: direct solve */
    or_cholesky_solve(nnc, h->chol, uc);
  } else {
    vcycle_level(h, l + 1, rc, uc);                           /* recursion from u = 0 */
  }
  or_prolong_add(n, uc, u);                                   /* u += P u^(l+1) */
  or_smooth(n, h->st[l], h->W[l], f, u, h->nu2);             /* post-smoothing */
  free(r);
  free(rc);
  free(uc);
}

void or_mg_vcycle(void* hv, const double* b, double* x) {
  or_mg* h = (or_mg*)hv;
  if (h->L == 1) {
    const int nn = h->n[0] * h->n[0];
    memcpy(x, b, sizeof(double) * nn);
    or_cholesky_solve(nn, h->chol, x);
    return;
  }
  vcycle_level(h, 0, b, x);
}

static double rel_residual(or_mg* h, const double* b, const double* x, double bnorm) {
  const int n = h->n[0], nn = n * n;
  double* r = (double*)malloc(sizeof(double) * nn);
  or_apply(n, h->st[0], x, r);
  double s = 0.0;
  for (int p = 0; p < nn; ++p) s += (b[p] - r[p]) * (b[p] - r[p]);
  free(r);
  return sqrt(s) / bnorm;
}

/* Repeat V-cycles until ||b - A x|| / ||b|| < rtol (the paper's stopping rule of Sec. 6.1,
   evaluation metrics) or max_cycles; hist[k] = relative residual after k cycles. */
int or_mg_solve(void* hv, const double* b, double* x, double rtol, int max_cycles, double* hist) {
  or_mg* h = (or_mg*)hv;
  const int nn = h->n[0] * h->n[0];
  double bn = 0.0;
  for (int p = 0; p < nn; ++p) bn += b[p] * b[p];
  bn = sqrt(bn);
  double rel = rel_residual(h, b, x, bn);
  if (hist) hist[0] = rel;
  int k = 0;
  while (k < max_cycles && !(rel < rtol)) {
    or_mg_vcycle(h, b, x);
    ++k;
    rel = rel_residual(h, b, x, bn);
    if (hist) hist[k] = rel;
  }
  return k;
}

/* ------------------------------------------------------------------------- */
/* Stencil-to-smoother network (Sec. 4.2, Fig. conv; layer widths of Sec. 6.2) */
/* ------------------------------------------------------------------------- */
/*
 * Per point, 9 input channels = the point's stencil divided by its centre coefficient
 * (zero outside the domain).  Three 3x3 convolution layers 9->7->5->3 with LeakyReLU
 * (slope 0.01), then a fully connected layer over the 3x3 window of the 3-channel map
 * (27 inputs) to the 9 taps of one 3x3 smoothing kernel.  The kernel applied at point
 * p is W_p = (omega * delta + out_p) / D_p, so a zero last layer gives weighted Jacobi.
 * Parameter layout: w1[7][9][3][3], w2[5][7][3][3], w3[3][5][3][3], wf[9][3][3][3].
 * bf16 != 0 rounds every weight and every layer input to bfloat16 before use.
 */
static const int HN_C[4] = {9, 7, 5, 3};
#define HN_SLOPE 0.01
#define HN_NPARAMS (7 * 9 * 9 + 5 * 7 * 9 + 3 * 5 * 9 + 9 * 3 * 9)

int or_hypernet_nparams(void) { return HN_NPARAMS; }

/* Round to the nearest bfloat16 (8 significant bits), ties to even. */
double or_bf16(double v) {
  if (v == 0.0 || !isfinite(v)) return v;
  int e;
  frexp(v, &e);
  const double scale = ldexp(1.0, 8 - e);
  return nearbyint(v * scale) / scale;
}

/* out[o][p] = sum_{c,ky,kx} w[o][c][ky][kx] in[c][p + (ky-1, kx-1)] (zero outside) */
static void conv3x3(int n, int cin, int cout, const double* w, const double* in, double* out) {
  const int nn = n * n;
  for (int o = 0; o < cout; ++o)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int c = 0; c < cin; ++c)
          for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx) {
              const int ii = i + ky - 1, jj = j + kx - 1;
              if (inside(n, ii, jj)) acc += w[((o * cin + c) * 3 + ky) * 3 + kx] * in[c * nn + ii * n + jj];
            }
        out[o * nn + i * n + j] = acc;
      }
}

typedef struct {
  double* a[4];   /* layer inputs a0 (normalised stencil), a1, a2, a3 (after activation, rounded) */
  double* z[3];   /* pre-activations of the three conv layers */
  double* w[4];   /* weights as used (rounded when bf16) */
} hn_tape;

static void hn_tape_free(hn_tape* t) {
  for (int k = 0; k < 4; ++k) { free(t->a[k]); free(t->w[k]); }
  for (int k = 0; k < 3; ++k) free(t->z[k]);
}

static const double* hn_layer_weights(const double* params, int layer) {
  switch (layer) {
    case 0: return params;
    case 1: return params + 7 * 9 * 9;
    case 2: return params + 7 * 9 * 9 + 5 * 7 * 9;
    default: return params + 7 * 9 * 9 + 5 * 7 * 9 + 3 * 5 * 9;
  }
}

static void hn_forward_tape(int n, const double* st, const double* params, int bf16,
                            hn_tape* t, double* out) {
  const int nn = n * n;
  static const int wsz[4] = {7 * 9 * 9, 5 * 7 * 9, 3 * 5 * 9, 9 * 3 * 9};
  for (int l = 0; l < 4; ++l) {
    t->w[l] = (double*)malloc(sizeof(double) * wsz[l]);
    const double* src = hn_layer_weights(params, l);
    for (int q = 0; q < wsz[l]; ++q) t->w[l][q] = bf16 ? or_bf16(src[q]) : src[q];
  }
  t->a[0] = (double*)malloc(sizeof(double) * 9 * nn);
  for (int c = 0; c < 9; ++c)
    for (int p = 0; p < nn; ++p) {
      const double v = st[c * nn + p] / st[4 * nn + p];
      t->a[0][c * nn + p] = bf16 ? or_bf16(v) : v;
    }
  for (int l = 0; l < 3; ++l) {
    const int cin = HN_C[l], cout = HN_C[l + 1];
    t->z[l] = (double*)malloc(sizeof(double) * cout * nn);
    t->a[l + 1] = (double*)malloc(sizeof(double) * cout * nn);
    conv3x3(n, cin, cout, t->w[l], t->a[l], t->z[l]);
    for (int q = 0; q < cout * nn; ++q) {
      const double z = t->z[l][q];
      const double a = z > 0.0 ? z : HN_SLOPE * z;
      t->a[l + 1][q] = bf16 ? or_bf16(a) : a;
    }
  }
  conv3x3(n, 3, 9, t->w[3], t->a[3], out); /* fully connected over the 3x3 window */
}

void or_hypernet_forward(int n, const double* st, const double* params, double omega,
                         int bf16, double* W) {
  const int nn = n * n;
  hn_tape t;
  memset(&t, 0, sizeof(t));
  double* out = (double*)malloc(sizeof(double) * 9 * nn);
  hn_forward_tape(n, st, params, bf16, &t, out);
  for (int k = 0; k < 9; ++k)
    for (int p = 0; p < nn; ++p)
      W[k * nn + p] = ((k == 4 ? omega : 0.0) + out[k * nn + p]) / st[4 * nn + p];
  free(out);
  hn_tape_free(&t);
}

/* Adjoint of conv3x3 with respect to its input (accumulate) and its weights (accumulate). */
static void conv3x3_backward(int n, int cin, int cout, const double* w, const double* in,
                             const double* gout, double* gin, double* gw) {
  const int nn = n * n;
  for (int o = 0; o < cout; ++o)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double g = gout[o * nn + i * n + j];
        if (g == 0.0) continue;
        for (int c = 0; c < cin; ++c)
          for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx) {
              const int ii = i + ky - 1, jj = j + kx - 1;
              if (!inside(n, ii, jj)) continue;
              const int widx = ((o * cin + c) * 3 + ky) * 3 + kx;
              gw[widx] += g * in[c * nn + ii * n + jj];
              if (gin) gin[c * nn + ii * n + jj] += g * w[widx];
            }
      }
}

/* dparams += d/dparams sum_{k,p} dW[k][p] W[k][p]; rounding is passed straight through. */
void or_hypernet_backward(int n, const double* st, const double* params, double omega,
                          int bf16, const double* dW, double* dparams) {
  (void)omega;
  const int nn = n * n;
  hn_tape t;
  memset(&t, 0, sizeof(t));
  double* out = (double*)malloc(sizeof(double) * 9 * nn);
  hn_forward_tape(n, st, params, bf16, &t, out);
  double* gout = (double*)malloc(sizeof(double) * 9 * nn);
  for (int k = 0; k < 9; ++k)
    for (int p = 0; p < nn; ++p) gout[k * nn + p] = dW[k * nn + p] / st[4 * nn + p];
  double* gw[4];
  for (int l = 0; l < 4; ++l) gw[l] = (double*)hn_layer_weights(dparams, l);
  double* ga3 = (double*)calloc(3 * nn, sizeof(double));
  conv3x3_backward(n, 3, 9, t.w[3], t.a[3], gout, ga3, gw[3]);
  double* gnext = ga3;
  for (int l = 2; l >= 0; --l) {
    const int cin = HN_C[l], cout = HN_C[l + 1];
    double* gz = (double*)malloc(sizeof(double) * cout * nn);
    for (int q = 0; q < cout * nn; ++q) gz[q] = gnext[q] * (t.z[l][q] > 0.0 ? 1.0 : HN_SLOPE);
    double* gin = l > 0 ? (double*)calloc(cin * nn, sizeof(double)) : NULL;
    conv3x3_backward(n, cin, cout, t.w[l], t.a[l], gz, gin, gw[l]);
    free(gz);
    free(gnext);
    gnext = gin;
  }
  free(gnext);
  free(out);
  free(gout);
  hn_tape_free(&t);
}

/* ------------------------------------------------------------------------- */
/* Convergence-theory training loss                                           */
/* ------------------------------------------------------------------------- */
/*
 * Two-grid error propagation with one pre- and one post-smoothing step and an exact
 * coarse solve (eq. twogrid, with the smoother applied before and after the coarse
 * correction): E = S C S, S = I - H A, C = I - P (P^T A P)^{-1} P^T A.  Following
 * eq. overalltrain with u_* = 0 and Thm. sbound, the loss over random vectors z_j is
 *     L = (1/Z) sum_j ||E z_j||^2 / n,     n = number of unknowns,
 * an estimate of ||E||_F^2 / n.  If dW != NULL, dW += dL/dW (per-point kernels).
 */
double or_twogrid_loss(int n, const double* st, const double* W, int nz, const double* z,
                       double* dW) {
  const int nn = n * n, nc = (n - 1) / 2, nnc = nc * nc;
  double* stc = (double*)malloc(sizeof(double) * 9 * nnc);
  or_rap(n, st, stc);
  double* Lc = (double*)malloc(sizeof(double) * (size_t)nnc * nnc);
  or_dense_matrix(nc, stc, Lc);
  or_cholesky(nnc, Lc);
  double *e0 = malloc(sizeof(double) * nn), *v0 = malloc(sizeof(double) * nn);
  double *e1 = malloc(sizeof(double) * nn), *e2 = malloc(sizeof(double) * nn);
  double *v2 = malloc(sizeof(double) * nn), *e3 = malloc(sizeof(double) * nn);
  double *tmp = malloc(sizeof(double) * nn), *tmp2 = malloc(sizeof(double) * nn);
  double* xc = malloc(sizeof(double) * nnc);
  double loss = 0.0;
  for (int s = 0; s < nz; ++s) {
    memcpy(e0, z + (size_t)s * nn, sizeof(double) * nn);
    /* e1 = e0 - H A e0 */
    or_apply(n, st, e0, v0);
    or_apply_H(n, W, v0, tmp);
    for (int p = 0; p < nn; ++p) e1[p] = e0[p] - tmp[p];
    /* e2 = e1 - P Ac^{-1} P^T A e1 */
    or_apply(n, st, e1, tmp);
    or_restrict(n, tmp, xc);
    or_cholesky_solve(nnc, Lc, xc);
    memcpy(e2, e1, sizeof(double) * nn);
    for (int p = 0; p < nn; ++p) tmp[p] = 0.0;
    or_prolong_add(n, xc, tmp);
    for (int p = 0; p < nn; ++p) e2[p] -= tmp[p];
    /* e3 = e2 - H A e2 */
    or_apply(n, st, e2, v2);
    or_apply_H(n, W, v2, tmp);
    for (int p = 0; p < nn; ++p) e3[p] = e2[p] - tmp[p];
    double sq = 0.0;
    for (int p = 0; p < nn; ++p) sq += e3[p] * e3[p];
    loss += sq / ((double)nz * nn);
    if (!dW) continue;
    /* adjoint: g3 = dL/de3 */
    double* g = e3; /* reuse */
    for (int p = 0; p < nn; ++p) g[p] = 2.0 * e3[p] / ((double)nz * nn);
    /* e3 = e2 - H v2: dW_p[k] -= g(p) v2(p + d_k) ; g2 = g - A H^T g */
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < 9; ++k) {
          const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
          if (inside(n, ii, jj)) dW[k * nn + i * n + j] -= g[i * n + j] * v2[ii * n + jj];
        }
    or_apply_HT(n, W, g, tmp);
    or_apply(n, st, tmp, tmp2);
    for (int p = 0; p < nn; ++p) g[p] -= tmp2[p];
    /* C^T = I - A P Ac^{-1} P^T */
    or_restrict(n, g, xc);
    or_cholesky_solve(nnc, Lc, xc);
    for (int p = 0; p < nn; ++p) tmp[p] = 0.0;
    or_prolong_add(n, xc, tmp);
    or_apply(n, st, tmp, tmp2);
    for (int p = 0; p < nn; ++p) g[p] -= tmp2[p];
    /* e1 = e0 - H v0 */
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < 9; ++k) {
          const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
          if (inside(n, ii, jj)) dW[k * nn + i * n + j] -= g[i * n + j] * v0[ii * n + jj];
        }
  }
  free(stc); free(Lc); free(e0); free(v0); free(e1); free(e2); free(v2); free(e3);
  free(tmp); free(tmp2); free(xc);
  return loss;
}

/*
 * The same objective after k two-grid cycles (eq. overalltrain with u_* = 0 and k cycles
 * of the solver, the form Algorithm 2 minimises over k): with E = S C S,
 *   loss = (1/nz) sum_j ||E^k z_j||^2 / n^2.
 * Forward: e_0 = z, e_{c+1} = E e_c, keeping A e_c and A (C S e_c) of every cycle.
 * Adjoint, cycles in reverse: g = dloss/de_{c+1} gives the two dW terms of cycle c
 * exactly as in or_twogrid_loss, and dloss/de_c = E^T g = S^T C^T S^T g feeds cycle c-1.
 */
double or_twogrid_loss_k(int n, const double* st, const double* W, int nz, const double* z, int ncycles,
                         double* dW) {
  const int nn = n * n, nc = (n - 1) / 2, nnc = nc * nc, K = ncycles;
  double* stc = (double*)malloc(sizeof(double) * 9 * nnc);
  or_rap(n, st, stc);
  double* Lc = (double*)malloc(sizeof(double) * (size_t)nnc * nnc);
  or_dense_matrix(nc, stc, Lc);
  or_cholesky(nnc, Lc);
  double* V0 = (double*)malloc(sizeof(double) * (size_t)K * nn); /* A e_c          */
  double* V2 = (double*)malloc(sizeof(double) * (size_t)K * nn); /* A (C S e_c)    */
  double *e = malloc(sizeof(double) * nn), *e1 = malloc(sizeof(double) * nn);
  double *g = malloc(sizeof(double) * nn), *tmp = malloc(sizeof(double) * nn), *tmp2 = malloc(sizeof(double) * nn);
  double* xc = malloc(sizeof(double) * nnc);
  double loss = 0.0;
  for (int s = 0; s < nz; ++s) {
    memcpy(e, z + (size_t)s * nn, sizeof(double) * nn);
    for (int c = 0; c < K; ++c) {
      double* v0 = V0 + (size_t)c * nn;
      double* v2 = V2 + (size_t)c * nn;
      /* pre-smoothing: e1 = e - H A e */
      or_apply(n, st, e, v0);
      or_apply_H(n, W, v0, tmp);
      for (int p = 0; p < nn; ++p) e1[p] = e[p] - tmp[p];
      /* coarse correction: e = e1 - P Ac^{-1} P^T A e1 */
      or_apply(n, st, e1, tmp);
      or_restrict(n, tmp, xc);
      or_cholesky_solve(nnc, Lc, xc);
      for (int p = 0; p < nn; ++p) tmp[p] = 0.0;
      or_prolong_add(n, xc, tmp);
      for (int p = 0; p < nn; ++p) e[p] = e1[p] - tmp[p];
      /* post-smoothing: e = e - H A e */
      or_apply(n, st, e, v2);
      or_apply_H(n, W, v2, tmp);
      for (int p = 0; p < nn; ++p) e[p] -= tmp[p];
    }
    double sq = 0.0;
    for (int p = 0; p < nn; ++p) sq += e[p] * e[p];
    loss += sq / ((double)nz * nn);
    if (!dW) continue;
    for (int p = 0; p < nn; ++p) g[p] = 2.0 * e[p] / ((double)nz * nn);
    for (int c = K - 1; c >= 0; --c) {
      const double* v0 = V0 + (size_t)c * nn;
      const double* v2 = V2 + (size_t)c * nn;
      /* post-smoothing of cycle c */
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < 9; ++k) {
            const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
            if (inside(n, ii, jj)) dW[k * nn + i * n + j] -= g[i * n + j] * v2[ii * n + jj];
          }
      or_apply_HT(n, W, g, tmp);
      or_apply(n, st, tmp, tmp2);
      for (int p = 0; p < nn; ++p) g[p] -= tmp2[p];
      /* C^T = I - A P Ac^{-1} P^T */
      or_restrict(n, g, xc);
      or_cholesky_solve(nnc, Lc, xc);
      for (int p = 0; p < nn; ++p) tmp[p] = 0.0;
      or_prolong_add(n, xc, tmp);
      or_apply(n, st, tmp, tmp2);
      for (int p = 0; p < nn; ++p) g[p] -= tmp2[p];
      /* pre-smoothing of cycle c */
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < 9; ++k) {
            const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
            if (inside(n, ii, jj)) dW[k * nn + i * n + j] -= g[i * n + j] * v0[ii * n + jj];
          }
      /* dloss/de_c = S^T g for the cycle before */
      if (c > 0) {
        or_apply_HT(n, W, g, tmp);
        or_apply(n, st, tmp, tmp2);
        for (int p = 0; p < nn; ++p) g[p] -= tmp2[p];
      }
    }
  }
  free(stc); free(Lc); free(V0); free(V2); free(e); free(e1); free(g); free(tmp); free(tmp2); free(xc);
  return loss;
}
