/*
 * mgcnn.h -- C ABI of the GB300 (sm_103a) learned-smoother multigrid library.
 *
 * Method: Huang, Li & Xi, "Learning optimal multigrid smoothers via neural networks"
 * (arXiv 2102.12071).  The library solves A u = f (Sec. 2, eq. Au=f; A symmetric positive
 * definite) on n x n interior grids of the unit square with homogeneous Dirichlet
 * boundaries by V-cycles (Algorithm 1) whose smoother is either weighted Jacobi
 * (Sec. 2.1) or the action H = M^{-1} produced per point by a convolutional network from
 * the operator stencil (Sec. 4.2), and it evaluates and differentiates the two-grid
 * convergence loss that trains that network (Sec. 3.2, eq. twogrid, Thm. sbound).
 *
 * Conventions shared by every entry point
 *   Grids      n x n interior points, n = 2^m - 1 (3 <= n <= 8191), row-major:
 *              element (i, j) at offset i*n + j, row i = y (north = +y), column j = x.
 *              Batched grids are contiguous [nprob][n][n].
 *   Stencils   9 coefficients, tap k = 3*(di+1) + (dj+1) is the coefficient of
 *              u(i+di, j+dj) in row (i, j) of A; k = 4 is the diagonal.  A stencil field
 *              is [9][n][n] (one stencil per point); taps that couple to points outside
 *              the interior must be zero (the field is exactly the rows of A).
 *   Kernels    per-point smoothing kernels use the stencil-field layout:
 *              (H v)(p) = sum_k W[k][p] * v(p + d_k), v = 0 outside the interior.
 *   Memory     every pointer documented "device" must point to memory of the current
 *              CUDA device; the caller owns every buffer, including the workspace.  The
 *              library allocates no device buffers; a context is a host struct that may
 *              also hold CUDA graphs of one V-cycle and a private capture stream (their
 *              runtime state is released by mg_destroy).
 *              Buffers must stay valid until the work queued on the stream completes.
 *   Streams    `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *              device work of a call is queued on it.  One context must not be used
 *              from two streams at once.
 *   Errors     every call returns an mg_status and never aborts; mg_last_error() gives
 *              a thread-local message for the last failing call.  A CUDA error is
 *              reported as MG_ERR_CUDA.
 */
#ifndef MGCNN_H
#define MGCNN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,   /* a size, pointer, kind or option is out of range        */
  MG_ERR_WORKSPACE = 2,     /* workspace too small or misaligned (needs 256 B)         */
  MG_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed             */
  MG_ERR_NOT_CONVERGED = 4, /* mg_solve hit max_cycles before rtol (results valid)     */
  MG_ERR_NUMERIC = 5,       /* NaN/Inf residual or a non-SPD coarsest operator         */
  MG_ERR_TIMEOUT = 6,       /* a bounded device-side wait for tile copies expired      */
  MG_ERR_UNSUPPORTED = 7    /* valid request outside what this build implements        */
} mg_status;

/* Operator of one problem (Sec. 3.1 eq. constant, Sec. 4 eq. vcoeff, Sec. 6.1 eq. pde). */
typedef enum {
  /* -div(K grad u), K = R(theta) diag(1, eps) R(theta)^T constant (the rotated anisotropic
     Laplacian of Sec. 6.1 with conductivity eps), bilinear (Q1) finite elements:
     9-point constant stencil.  Uses eps (> 0) and theta; data must be NULL. */
  MG_PROBLEM_ROTATED = 0,
  /* constant 9-point stencil given by the caller: data = HOST float[9] (tap layout above). */
  MG_PROBLEM_STENCIL = 1,
  /* -div(a grad u) with a constant per cell, 5-point stencil whose edge weights are the
     mean of the two cells sharing the edge: data = DEVICE float[(n+1)*(n+1)], cell (ci, cj)
     spans mesh rows ci..ci+1 and columns cj..cj+1 (interior unknown (i,j) = mesh node
     (i+1, j+1)); values must be positive. */
  MG_PROBLEM_VARCOEF5 = 2,
  /* per-point 9-point stencil field given by the caller: data = DEVICE float[9*n*n]. */
  MG_PROBLEM_FIELD = 3
} mg_problem_kind;

typedef struct {
  int n;              /* interior points per side, 2^m - 1                          */
  int kind;           /* mg_problem_kind                                            */
  double eps;         /* MG_PROBLEM_ROTATED: conductivity (eps in (0, 1] typical)   */
  double theta;       /* MG_PROBLEM_ROTATED: angle of anisotropy, radians           */
  const float* data;  /* see mg_problem_kind; copied during mg_setup                */
} mg_problem;

typedef enum {
  MG_SMOOTH_JACOBI = 0, /* weighted Jacobi, H = omega D^{-1} (Sec. 2.1)              */
  MG_SMOOTH_CNN = 1     /* per-point 3x3 kernels from the stencil network (Sec. 4.2)  */
} mg_smoother_kind;

typedef struct {
  int smoother;     /* mg_smoother_kind                                               */
  int nu1, nu2;     /* pre-/post-smoothing steps per level (Algorithm 1), 1..8: the
                       first pre-smoothing step is e = H r from e = 0, every further
                       step e += H (r - A e).  Other than 1 only with MG_SMOOTH_JACOBI or
                       MG_NET_LINEAR (MG_ERR_UNSUPPORTED otherwise); such contexts run the
                       levels above 63 in batched level kernels, not the fused tiles
                       (Sec. 6: six Jacobi steps per smoothing equal the six convolutions
                       of the linear network in cost)                                   */
  float omega;      /* Jacobi weight (2/3 in the paper, Sec. 6.1); also the Jacobi part
                       of the network output W = (omega*delta + NN)/D                   */
  int coarsest_n;   /* stop coarsening at this size (this build: 3)                  */
  int conv_bf16;    /* 1: network weights and activations rounded to bfloat16, FP32
                       accumulation; 0: FP32 throughout                                 */
  int cluster_tail; /* 1: the levels below the finest of side <= 63 (network smoothers
                       on fine grids of side >= 1023; row bands on the levels above 15)
                       or <= 127 (otherwise; bands above 31) run in one cluster of 8 CTAs
                       per problem with every vector in
                       shared memory, where the device can hold such a cluster, and the
                       levels above in tiled kernels; 0: the levels of side <= 63 run in
                       one CTA per problem and the levels above in tiled kernels.  Both
                       compute the same cycle; the choice only changes how it is laid out
                       on the GPU.  Problems of side <= 63 always run in one CTA each.   */
  int train_cycles;     /* training only (mg_train_*): the most two-grid cycles k the loss
                           may span, workspace reserved for (0 or 1: one cycle; <= 16)   */
  int train_checkpoint; /* training only: 1 keeps just each cycle's input vectors and
                           recomputes the cycle's operator products in the backward pass
                           (one vector set per cycle instead of three)                   */
  int net_levels;       /* MG_SMOOTH_CNN: 0 or 1 -- one network for every level; k > 1 --
                           net_params holds k parameter sets and level l uses set
                           min(l, k - 1) (per-level smoothers H^(l), Algorithm 2)        */
  int smoother_transpose; /* 1: every level smooths with H^T instead of H (per-point
                           problems, or MG_NET_LINEAR: the chain reversed with mirrored
                           kernels, or MG_NET_CONV3: the stack reversed with each kernel
                           transposed), so a V-cycle of this context applies M^T when the
                           context without it applies M: the adjoint coarse solve of
                           mg_train_step_coarse                                          */
  int net_arch;         /* MG_SMOOTH_CNN: mg_net_arch; parameter sets hold
                           mg_net_param_count(net_arch) floats                           */
  int net_per_problem;  /* MG_NET_LINEAR only: 1 -- net_params holds max(1, net_levels)
                           sets for each problem of the batch, [nprob][sets][54] in batch
                           order (Sec. 6 trains one smoother per problem); 0 -- one group
                           of sets shared by every problem                               */
  int tile_shape;       /* mg_tile_shape: how the down-sweep kernels of the levels above
                           the coarse tail cover a level (the up-sweeps always use 32 x 32
                           tiles).  Every shape computes the same cycle (up to the order of
                           FP32 roundings); it only changes the work per CTA, so the fastest
                           one depends on the grid size, the smoother and the batch: strips
                           pay off when many problems fill the GPU, tiles when few do.     */
} mg_options;

typedef enum {
  MG_TILE_DEFAULT = 0,    /* MG_TILE_PSTRIP (which leaves the batches it does not cover
                             to MG_TILE_32x32)                                          */
  MG_TILE_32x32 = 1,      /* one 32 x 32 block of points per CTA, 3x3 windows in shared
                             memory                                                     */
  MG_TILE_STRIP4x32 = 2,  /* warp strips: a warp owns 26 columns and walks down the rows,
                             neighbours by warp shuffles; CTAs of 4 strips x 32 rows    */
  MG_TILE_STRIP8x64 = 3,  /* ... CTAs of 8 strips x 64 rows                             */
  MG_TILE_STRIP8x32 = 4,  /* ... CTAs of 8 strips x 32 rows                             */
  MG_TILE_PSTRIP = 5      /* paired warp strips (constant stencils with the Jacobi or
                             network smoother; other batches use 32 x 32 tiles): lane k
                             holds a pair of adjacent columns in packed FP32, a warp owns
                             60 columns and walks down a height chosen per launch so that
                             all walks fill about one wave, its rows arriving in 8-row
                             copies through a ring of its own; bit-identical to 32 x 32 */
} mg_tile_shape;

typedef enum {
  MG_NET_CONV = 0, /* 3x3 convolutions 9->7->5->3 and a 27->9 layer (Sec. 4.2, 1 260 params) */
  MG_NET_FC = 1,   /* fully connected 81->40->40->40->9 on the 3x3 neighbourhood's stencils
                      (Sec. 4.2 parameterisation with fully connected layers, Sec. 6.2:
                      6 800 params)                                                      */
  MG_NET_LINEAR = 2, /* the shared-kernel linear smoother of Sec. 6 (eq.
                      full-coarsening-smoother): H = f5(f4(f3(f2(f1(.))))) + f6, each f_k a
                      3x3 convolution (tap layout above) whose input is zero outside the
                      grid, the same six kernels at every point of every problem of a
                      context.  A parameter set is float[6][9] = (f1 .. f5, f6), 54 params;
                      the network has no input: its weights are the smoother.  Weighted
                      Jacobi is f1..f4 = identity (tap 4 = 1), f5 = 0, f6 = omega/D at tap 4.
                      Any stencil kind.                                                  */
  MG_NET_CONV3 = 3, /* the convolutional network of MG_NET_CONV with 27 outputs per point:
                      three 3x3 kernels applied as a stack H v = K3(K2(K1 v)), each
                      layer's input zero outside the grid (Sec. 4, Sec. 4.2: k = 3),
                      K1 = (omega delta + out_1)/D, K2 = delta + out_2, K3 = delta + out_3;
                      last layer wf[27][3][3][3] (row 9k + t: tap t of kernel k+1), 1 746
                      params.  FP32 only; solve, V-cycle, FGMRES, mg_train_step and
                      (with smoother_transpose for the adjoint) mg_train_step_coarse;
                      mg_smoother_apply and mg_get_kernels refuse it.  Levels above 63
                      run in the batched level kernels.                                  */
  MG_NET_CONV_SHARED = 4 /* the network of MG_NET_CONV with one 3x3 kernel per output
                      channel of each convolution, applied to every input channel of the
                      layer (out_o = k_o * sum_c in_c): the 378-parameter count of
                      Sec. 6.2, (7 + 5 + 3) * 9 + 27 * 9.  Layout: k1[7][3][3],
                      k2[5][3][3], k3[3][3][3], wf[9][3][3][3].  It is MG_NET_CONV with
                      w[o][c] = k_o for every c; the library expands each set on the
                      device and sums the dense gradient over c.  Everything MG_NET_CONV
                      supports.                                                          */
} mg_net_arch;

typedef struct mg_ctx mg_ctx;
typedef struct mg_train_ctx mg_train_ctx;

/* ---------------------------------------------------------------- hierarchy ---- */

/* Bytes of device workspace mg_setup needs for this batch (0 if the arguments are
   invalid; mg_last_error() says why).  All problems of one batch must share n and be
   either all constant-stencil (ROTATED/STENCIL) or all per-point (VARCOEF5/FIELD). */
size_t mg_workspace_size(const mg_problem* problems, int nprob, const mg_options* opts);

/* Builds the multigrid hierarchy of Algorithm 1 for nprob problems on `stream`:
   level-0 stencils (Sec. 6.1 eq. pde / Sec. 4), Galerkin coarse operators P^T A P
   (Sec. 2.2) with full coarsening and bilinear P (Sec. 6.1, Fig. full_coarsening) down to
   coarsest_n, the FP64 inverse of the coarsest operator, and -- for
   MG_SMOOTH_CNN -- the per-point smoothing kernels of every smoothed level from the
   network with parameters net_params (DEVICE, max(1, net_levels) sets of
   mg_net_param_count(net_arch) floats, read during this call only; NULL for Jacobi;
   MG_NET_LINEAR copies its sets as the levels' smoothers).  workspace: DEVICE, >= mg_workspace_size bytes, 256-byte
   aligned, owned by the caller and used exclusively by this context until mg_destroy.
   On success *out receives a host handle. */
mg_status mg_setup(const mg_problem* problems, int nprob, const mg_options* opts,
                   const float* net_params, void* workspace, size_t ws_bytes,
                   void* stream, mg_ctx** out);

/* Releases the host handle (the workspace stays the caller's). NULL is ignored. */
void mg_destroy(mg_ctx* ctx);

int mg_num_levels(const mg_ctx* ctx);          /* levels including the coarsest      */
int mg_level_n(const mg_ctx* ctx, int level);  /* side of level `level`, 0 if invalid */

/* Copies the stencil field of (prob, level) to out (DEVICE float[9*n_l*n_l]). */
mg_status mg_get_stencil(const mg_ctx* ctx, int prob, int level, float* out, void* stream);

/* Copies the per-point smoothing kernels H of (prob, level) to out (DEVICE
   float[9*n_l*n_l]), expanded to one 3x3 kernel per point (Jacobi: omega/D at tap 4).
   MG_NET_LINEAR has no such kernels: MG_ERR_UNSUPPORTED. */
mg_status mg_get_kernels(const mg_ctx* ctx, int prob, int level, float* out, void* stream);

/* Weighted-Jacobi or CNN smoothing on one level of one problem (eq. iteration):
   nsteps times u <- u + H (f - A u).  f, u: DEVICE float[n_l*n_l].  Uses the context's
   level-`level` work vectors as scratch. */
mg_status mg_smoother_apply(mg_ctx* ctx, int prob, int level, const float* f, float* u,
                            int nsteps, void* stream);

/* ------------------------------------------------------------------ solving ---- */

/* One V-cycle (Algorithm 1) on every problem: x <- x + V(b - A x), where the iterate
   x = x_hi + x_lo is an unevaluated float-float pair so the outer residual can reach 1e-8.
   b, x_hi: DEVICE float[nprob*n*n]; x_lo: DEVICE float[nprob*n*n] or NULL (then x_lo is
   taken as zero and not written); rel_res: DEVICE float[nprob] or NULL, receives
   ||b - A x||_2 / ||b||_2 after the cycle.  The cycle runs on the error equation A e = r
   in FP32; the outer residual is evaluated in compensated (float-float) arithmetic. */
mg_status mg_vcycle(mg_ctx* ctx, const float* b, float* x_hi, float* x_lo, float* rel_res,
                    void* stream);

/* Repeats V-cycles until ||b - A x||_2 / ||b||_2 < rtol (the stopping rule of Sec. 6.1,
   evaluation metrics) or max_cycles cycles, per problem.  b, x_hi, x_lo as for mg_vcycle
   (x_hi holds the initial guess; x_lo NULL means a zero low part kept in the workspace).
   hist: HOST double[nprob*(max_cycles+1)] or NULL; row p receives the relative residual
   after 0, 1, ... cycles (entries past cycles[p] are left untouched).  cycles: HOST
   int[nprob] or NULL, receives the cycle count per problem.  Blocks the calling thread
   until `stream` has finished the solve.  Returns MG_ERR_NOT_CONVERGED if any problem
   stopped at max_cycles, MG_ERR_NUMERIC on a NaN/Inf residual. */
mg_status mg_solve(mg_ctx* ctx, const float* b, float* x_hi, float* x_lo, double rtol,
                   int max_cycles, double* hist, int* cycles, void* stream);

/* Solves of several independent batches at once (no counterpart in the paper; its
   experiments solve problems one by one): the same as mg_solve on every context, for
   batches of different sizes or stencil kinds, which one context cannot hold.  Context k
   runs on streams[k] (NULL array or entry: the default stream) with its arrays b[k],
   x_hi[k], x_lo[k] (x_lo NULL or an entry NULL: zero low parts) and cycles[k] (NULL array
   or entry: not reported; else HOST int[nprob of context k]).  The host polls the
   streams and issues a context's next chunk of cycles as soon as its previous chunk is
   done, so the batches' kernels overlap on the GPU and no context waits for another.
   The contexts must be distinct.  Blocks until all have finished.  The per-problem
   outcomes (MG_ERR_NOT_CONVERGED, MG_ERR_NUMERIC, MG_ERR_TIMEOUT) stop no other context:
   the first non-OK one in context order is returned.  A CUDA or argument error returns at
   once, after waiting for every context's stream. */
mg_status mg_solve_multi(mg_ctx* const* ctxs, int nctx, const float* const* b, float* const* x_hi,
                         float* const* x_lo, double rtol, int max_cycles, int* const* cycles,
                         void* const* streams);

/* ------------------------------------------------------- Krylov acceleration ---- */

/* Bytes of device workspace mg_fgmres needs for this context and restart length
   (1 <= restart <= 200; 0 on invalid arguments). */
size_t mg_fgmres_workspace_size(const mg_ctx* ctx, int restart);

/* Flexible GMRES(restart) with one V(1,1) cycle of ctx (its smoother) as the right
   preconditioner (Sec. 6.4), for every problem of the batch: Arnoldi on A M keeping the
   preconditioned directions z_j = M v_j, classical Gram-Schmidt with one
   re-orthogonalisation, Givens rotations, x = x_0 + Z y.  A problem stops when the
   least-squares residual estimate reaches ||b - A x|| / ||b|| < rtol or after max_iters
   preconditioned steps in all.  b, x_hi, x_lo as for mg_solve (x_hi + x_lo the initial
   guess in and the float-float solution out; x_lo NULL: zero low part kept in the
   workspace); every restart evaluates b - A x in compensated arithmetic.  hist: HOST
   double[nprob * (max_iters + 1)] or NULL, row p the relative residual estimate after
   0, 1, ... steps; iters: HOST int[nprob] or NULL, steps per problem.  workspace: DEVICE,
   >= mg_fgmres_workspace_size bytes, 256-byte aligned, caller-owned.  Returns
   MG_ERR_NOT_CONVERGED if the final (compensated) residual of a problem is >= rtol.
   Blocks the calling thread; uses ctx's workspace (no solve may run on ctx meanwhile). */
mg_status mg_fgmres(mg_ctx* ctx, const float* b, float* x_hi, float* x_lo, int restart,
                    double rtol, int max_iters, void* workspace, size_t ws_bytes,
                    double* hist, int* iters, void* stream);

/* ------------------------------------------------------------ network (a3) ---- */

/* Number of network parameters: 3x3 convolutions 9->7->5->3 (no bias) and the layer
   from the 3x3 window of the 3-channel map (27 inputs) to the 9 kernel taps
   (Sec. 4.2 and the layer sizes of Sec. 6.2).  Layout: w1[7][9][3][3], w2[5][7][3][3],
   w3[3][5][3][3], wf[9][3][3][3]; LeakyReLU slope 0.01 after each convolution. */
int mg_net_nparams(void);

/* Parameters of a network architecture (mg_net_arch); 0 for an unknown one.  The standalone
   mg_net_forward below takes the MG_NET_CONV layout. */
int mg_net_param_count(int arch);

/* Network inference on nprob stencil fields (DEVICE float[nprob][9][n][n]): per point,
   input channel c = st[c]/st[4] (zero outside the grid), output kernel
   W = (omega*delta_4 + NN)/st[4] written to W (DEVICE float[nprob][9][n][n]).
   params: DEVICE float[mg_net_nparams()]. */
mg_status mg_net_forward(int n, int nprob, const float* fields, const float* params,
                         float omega, int conv_bf16, float* W, void* stream);

/* The same for the fully connected network (MG_NET_FC): per point the 81 values of its
   3x3 neighbourhood, feature 9 m + c = tap c of the neighbour at offset m (row-major
   3x3 offsets) divided by that neighbour's diagonal, zero outside the grid; layers
   81->40->40->40->9 (weights [out][in] consecutively, no biases), LeakyReLU 0.01 after
   the hidden layers, W = (omega*delta_4 + out)/diag.  params: DEVICE float[6800]. */
mg_status mg_net_fc_forward(int n, int nprob, const float* fields, const float* params,
                            float omega, int bf16, float* W, void* stream);

/* --------------------------------------------------------- training (a11-a12) ---- */

/* Bytes of device workspace for mg_train_setup (0 on invalid arguments). */
size_t mg_train_workspace_size(const mg_problem* problems, int nprob, int nvec,
                               const mg_options* opts);

/* Prepares a training batch of nprob problems (all of one size n >= 7, any kinds of
   mg_problem_kind), nvec random vectors each: stencil fields, the two-grid Galerkin
   operator P^T A P and its FP64 banded Cholesky factor.  workspace: DEVICE, caller-owned. */
mg_status mg_train_setup(const mg_problem* problems, int nprob, int nvec,
                         const mg_options* opts, void* workspace, size_t ws_bytes,
                         void* stream, mg_train_ctx** out);

void mg_train_destroy(mg_train_ctx* ctx);

/* Loss and gradient of the two-grid convergence objective (eq. twogrid with one pre- and
   one post-smoothing step, eq. overalltrain with u_* = 0, Thm. sbound), after k cycles:
     loss = (1/nprob) sum_b (1/nvec) sum_j || (S C S)^k z_bj ||^2 / n^2,
     S = I - H A,  C = I - P (P^T A P)^{-1} P^T A,
   with H the network's per-point kernels for problem b (MG_NET_CONV, MG_NET_CONV_SHARED,
   MG_NET_FC), the stack K3 K2 K1 of MG_NET_CONV3 (FP32 only) or the linear chain of
   MG_NET_LINEAR, and k set by mg_train_set_cycles
   (default: train_cycles of the setup).  z: DEVICE float[nprob][nvec][n][n] (the random
   vectors, supplied by the caller), params and grad_out: DEVICE
   float[mg_net_param_count(net_arch of the setup)] (grad_out overwritten with dloss/dparams,
   the adjoint through all k cycles; may be NULL), loss_out: DEVICE float[1]. */
mg_status mg_train_step(mg_train_ctx* ctx, const float* params, const float* z,
                        float* grad_out, float* loss_out, void* stream);

/* mg_train_step with the coarse solve of every cycle replaced by one V(1,1) cycle from
   zero of an already-trained hierarchy below: the objective of Algorithm 2 at one level,
     E = S (I - P M P^T A) S,  M = one V-cycle of `coarse` (its smoothers H^(l+1..)),
   and the adjoint through M^T, one V-cycle of `coarse_t`.  coarse and coarse_t are
   contexts of the nprob coarse operators P^T A P of this batch (mg_train_get_coarse_field),
   in batch order, with (n - 1) / 2 <= 63 points per side, built with the same smoother
   parameters; coarse_t with smoother_transpose = 1.  Other arguments as mg_train_step. */
mg_status mg_train_step_coarse(mg_train_ctx* ctx, const float* params, const float* z,
                               mg_ctx* coarse, mg_ctx* coarse_t, float* grad_out,
                               float* loss_out, void* stream);

/* The Galerkin coarse operator P^T A P of problem `prob` of the batch as a per-point
   stencil field: out DEVICE float[9][nc][nc], nc = (n - 1) / 2. */
mg_status mg_train_get_coarse_field(const mg_train_ctx* ctx, int prob, float* out, void* stream);

/* Number of two-grid cycles k of the following mg_train_step calls, 1 <=
   max(1, train_cycles of the setup); Algorithm 2 draws k uniformly per step.  Host-only. */
mg_status mg_train_set_cycles(mg_train_ctx* ctx, int cycles);

/* ------------------------------------------------- solving without a workspace ---- */

/* Limits of mg_solve_small_static: its scratch is a fixed device array of
   MG_STATIC_SCRATCH_BYTES inside the library, enough for MG_STATIC_MAX_PROBLEMS problems
   of at most MG_STATIC_MAX_N points per side. */
#define MG_STATIC_MAX_PROBLEMS 16
#define MG_STATIC_MAX_N 63
#define MG_STATIC_SCRATCH_BYTES (512 * 1024)

/* The paper has no counterpart to this call; it exists for callers that cannot allocate
   device memory: plugins whose host framework's caching allocator owns the GPU memory,
   control loops with a fixed memory budget that must not risk an allocation failure while
   running, and latency-bound code that cannot pay for cudaMalloc/cudaFree (they may
   synchronise the device).  It performs what mg_workspace_size + mg_setup + mg_solve do
   for a batch of small constant-stencil problems (MG_PROBLEM_ROTATED or MG_PROBLEM_STENCIL,
   all of one size n = 2^m - 1 <= MG_STATIC_MAX_N, at most MG_STATIC_MAX_PROBLEMS of them)
   with weighted-Jacobi V(1,1) cycles down to a 3x3 grid, but allocates nothing: its
   scratch is a device array of MG_STATIC_SCRATCH_BYTES compiled into the library, held by
   every GPU that loads the library until the process exits.  Larger requests fail with
   MG_ERR_INVALID_ARG (other smoothers or options: MG_ERR_UNSUPPORTED).
   Arguments, outputs and return codes are those of mg_solve (b, x_hi, x_lo DEVICE
   [nprob][n][n], x_lo may be NULL; hist, cycles HOST or NULL); opts must ask for
   MG_SMOOTH_JACOBI, nu1 = nu2 = 1, coarsest_n = 3.  Every call looks up the array's device
   address on the current device (a host-side query).  Every call reuses the same array
   and resets what must start from zero; calls whose GPU work overlaps (two threads, or two
   streams) race on it and must be serialised by the caller.  Blocks the calling thread
   until the solve has finished (it reads the control blocks back after each chunk of
   cycles). */
mg_status mg_solve_small_static(const mg_problem* problems, int nprob, const mg_options* opts,
                                const float* b, float* x_hi, float* x_lo, double rtol,
                                int max_cycles, double* hist, int* cycles, void* stream);

/* ------------------------------------------------------------ measurement ---- */

/* Optional CUDA-event timing of individual kernel launches on the launching stream, for
   measurement tools; solving does not need it.  mg_profile_enable resets all counters and
   turns timing on (enable != 0) or off.  Timings are collected whenever mg_solve
   synchronises and by mg_profile_read (which requires the stream to be idle).
   kernel_class: 0 outer residual, 1 down-sweep of level 0, 2 up-sweep of level 0 (with the
   iterate update), 3 one-CTA coarse tail / small-problem solve, 4 down-sweeps of levels >= 1,
   5 up-sweeps of levels >= 1; -1 returns in *launches the number of kernels this context
   launched since the last reset (timing or not). */
mg_status mg_profile_enable(mg_ctx* ctx, int enable);

/* Per-problem timing of the last mg_solve or mg_solve_multi of ctx (the paper has no
   counterpart; used to report time to tolerance in mixed batches): start_ns[p], the GPU
   global timer in nanoseconds when the norm of b_p was formed at the start of the solve,
   and done_ns[p], when the stopping test that ended problem p ran (0 if it had not ended).
   Both HOST arrays of nprob entries; the timer is common to all SMs of the device, so
   stamps of several contexts solved together compare directly.  Host-only. */
mg_status mg_solve_times(const mg_ctx* ctx, unsigned long long* start_ns, unsigned long long* done_ns);

/* Test setting for failure detection (the paper has no counterpart): with on != 0 the
   following solves and cycles of ctx make the first bounded wait for every tile's copies
   give up at once, so the expiry path runs: the wait for the copies still in flight keeps
   its full bound (they land before the CTA exits), the problem is marked timed out, and
   mg_solve / mg_vcycle report MG_ERR_TIMEOUT.  It concerns the tiled levels only (n > 63);
   on = 0 restores normal solves.  Host-only; takes effect at the next solve or cycle. */
mg_status mg_debug_short_wait(mg_ctx* ctx, int on);

/* Test setting for the paired strips (tile_shape MG_TILE_PSTRIP): the least number of rows
   a warp's walk must have for the strips to take a level's down-sweep launch; launches
   with shorter walks (few problems active, small levels) run the 32 x 32 tiles, whose
   results are bit-identical.  Default 32; 0 sends every launch of a constant-stencil level
   with the Jacobi or network smoother to the strips.  rows < 0: MG_ERR_INVALID_ARG.
   Host-only; takes effect at the next solve or cycle. */
mg_status mg_debug_strip_rows(mg_ctx* ctx, int rows);
mg_status mg_profile_read(mg_ctx* ctx, int kernel_class, double* total_ms, long long* launches);

/* ------------------------------------------------------------------- misc ---- */

/* Interior Q1 stencil of MG_PROBLEM_ROTATED, rounded to float (host, no device work). */
mg_status mg_rotated_stencil(double eps, double theta, float out[9]);

const char* mg_status_string(mg_status s);
const char* mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MGCNN_H */
