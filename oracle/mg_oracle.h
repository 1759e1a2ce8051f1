/*
 * mg_oracle.h -- FP64 CPU oracle for the learned-smoother multigrid method of
 * Huang, Li & Xi, "Learning optimal multigrid smoothers via neural networks"
 * (arXiv 2102.12071).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct restatement
 * of the method used to check the CUDA path.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header or
 * constant with the CUDA library and the CUDA library never calls it.
 *
 * Conventions (all functions):
 *   - grids are n x n interior points of the unit square, homogeneous Dirichlet;
 *     index p = i*n + j, i = row = y (north = +y), j = column = x;
 *   - a 9-point stencil s[k] holds the coefficient of u(i+di, j+dj) in row (i, j)
 *     of A, with k = 3*(di+1) + (dj+1); k = 4 is the centre;
 *   - a stencil field st[k*n*n + p] stores one such stencil per point; couplings
 *     to points outside the interior are zero (the field is exactly the rows of A);
 *   - per-point smoothing kernels W use the same layout: (H v)(p) = sum_k W[k][p] v(p+d_k).
 */
#ifndef MG_ORACLE_H
#define MG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- discretisations (Sec. 3.1 eq. constant, Sec. 4 eq. vcoeff, Sec. 6.1 eq. pde) ---- */
void or_fe_q1_field(int n, const double* kxx, const double* kxy, const double* kyy,
                    int per_cell, double* st);
void or_q1_rotated_stencil(double eps, double theta, double s[9]);
void or_fd_rotated_stencil(double xi, double theta, double s[9]);
void or_paper9_field(int n, const double* g_cells, double* st);
void or_varcoef5_field(int n, const double* a_cells, double* st);
void or_const_field(int n, const double s[9], double* st);

/* ---- operators (Sec. 2.2, eq. twogrid; Sec. 6.1 transfer stencils) ---- */
void or_apply(int n, const double* st, const double* x, double* y);
void or_restrict(int n, const double* r, double* rc);
void or_prolong_add(int n, const double* ec, double* e);
void or_rap(int n, const double* st, double* stc);
void or_dense_matrix(int n, const double* st, double* A);

/* ---- smoothers (Sec. 2.1 eq. iteration; Sec. 4) ---- */
void or_jacobi_kernels(int n, const double* st, double omega, double* W);
void or_apply_H(int n, const double* W, const double* v, double* y);
void or_apply_HT(int n, const double* W, const double* v, double* y);
void or_smooth(int n, const double* st, const double* W, const double* f, double* u, int nsteps);
void or_gauss_seidel(int n, const double* st, const double* f, double* u);

/* ---- dense Cholesky for the coarsest solve ---- */
int  or_cholesky(int m, double* A);
void or_cholesky_solve(int m, const double* L, double* b);

/* ---- hierarchy, V-cycle and solve (Algorithm 1) ---- */
void* or_mg_create(int n, const double* st0, int coarsest_n, int nu1, int nu2);
void  or_mg_destroy(void* h);
int   or_mg_levels(void* h);
int   or_mg_n(void* h, int level);
void  or_mg_get_field(void* h, int level, double* st);
void  or_mg_get_kernels(void* h, int level, double* W);
void  or_mg_set_kernels(void* h, int level, const double* W);
void  or_mg_set_jacobi(void* h, double omega);
int   or_mg_set_cnn(void* h, const double* params, double omega, int bf16);
void  or_mg_vcycle(void* h, const double* b, double* x);
int   or_mg_solve(void* h, const double* b, double* x, double rtol, int max_cycles, double* hist);

/* ---- stencil-to-smoother network (Sec. 4.2, Fig. conv; sizes of Sec. 6.2) ---- */
int  or_hypernet_nparams(void);
double or_bf16(double v);
void or_hypernet_forward(int n, const double* st, const double* params, double omega,
                         int bf16, double* W);
void or_hypernet_backward(int n, const double* st, const double* params, double omega,
                          int bf16, const double* dW, double* dparams);

/* ---- convergence-theory loss (eq. twogrid, eq. overalltrain, Thm. sbound) ---- */
double or_twogrid_loss(int n, const double* st, const double* W, int nz, const double* z,
                       double* dW);
/* the same objective after ncycles >= 1 two-grid cycles: (1/nz) sum ||(S C S)^k z||^2 / n^2 */
double or_twogrid_loss_k(int n, const double* st, const double* W, int nz, const double* z,
                         int ncycles, double* dW);

#ifdef __cplusplus
}
#endif
#endif
