// mg_internal.h -- launchers shared between the C-ABI layer and the kernel files.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "mg_common.cuh"

struct mg_ctx;  // the library's context (mgcnn.h)

namespace mg {

// Kernel classes timed by the optional event profiler.
enum { PK_RESIDUAL = 0, PK_DOWN0 = 1, PK_UP0 = 2, PK_TAIL = 3, PK_DOWN = 4, PK_UP = 5, PK_NCLASS = 6 };

// CUDA-event timing of individual launches on the launching stream; events are reused
// after each collect() (called once the stream has been synchronised).
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> cls;
  int used = 0;
  double ms[PK_NCLASS] = {};
  long long count[PK_NCLASS] = {};
  long long launches = 0;  // every kernel launch, profiled or not

  void begin(int c, cudaStream_t s) {
    if (!on) return;
    if ((int)cls.size() <= used) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      ev.push_back(a);
      ev.push_back(b);
      cls.push_back(0);
    }
    cls[used] = c;
    cudaEventRecord(ev[2 * used], s);
  }
  void end(cudaStream_t s) {
    if (!on) return;
    cudaEventRecord(ev[2 * used + 1], s);
    ++used;
  }
  void collect() {
    for (int i = 0; i < used; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
        ms[cls[i]] += t;
        count[cls[i]] += 1;
      }
    }
    used = 0;
  }
  void reset() {
    collect();
    for (int c = 0; c < PK_NCLASS; ++c) { ms[c] = 0; count[c] = 0; }
    launches = 0;
  }
  ~Profiler() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// TMA descriptors of the tiled level kernels (mg_tiles.cu); every map is a 3-D tensor
// {x, y, problem} over one pitched level array of the whole batch.
struct ResMaps {
  CUtensorMap xh, xl, b;
};
struct DownMaps {
  CUtensorMap r;   // load: r_l with halo
  CUtensorMap e;   // store: e_l on the tile
  CUtensorMap rc;  // store: r_{l+1} on the coarse tile
};
struct UpMaps {
  CUtensorMap e, r, ec, xh, xl;
};
// level 0: up-sweep, update of x and the residual of the new iterate in one kernel
struct Up0Maps {
  CUtensorMap e, r, ec;  // boxes one point wider than UpMaps' (the update covers a halo)
  ResMaps x;             // x_hi, x_lo with a one-point halo, b
};
struct TileMaps {
  ResMaps res;
  DownMaps down[MG_MAXL];
  UpMaps up[MG_MAXL];
  Up0Maps up0;
  CUtensorMap down0_rb, up0_rb;  // level-0 residual loads of odd cycles (from r0b)
  ResMaps resb;                  // x loads of odd cycles (from xh0b, xl0b)
  // strip layouts (mg_strip.cu): the down-sweep's r block of each tiled level, and level
  // 0's from r0b on odd cycles
  CUtensorMap sr[MG_MAXL];
  CUtensorMap sr0b;
};

// base pointers of the pitched level arrays (all problems of a level contiguous)
struct LevelArrays {
  int n[MG_MAXL], pitch[MG_MAXL];
  float* r[MG_MAXL];
  float* e[MG_MAXL];
  float* f[MG_MAXL];      // final corrections of the tiled levels >= 1 (LevelDev::f)
  float *xh0, *xl0, *b0;  // the iterate pair and right-hand side, pitched like level 0
  float *xh0b, *xl0b;     // second iterate pair: cycles alternate the two pairs
  float* r0b;             // second level-0 residual: cycles alternate r[0] and r0b
};

// TMA maps of the linear smoother's tiled chain (mg_linear.cu): the vector a smoothing
// applies H to, with the chain's five-point halo
struct LinMaps {
  CUtensorMap r0a, r0b;    // level 0: the two residual arrays (cycle parity)
  CUtensorMap r[MG_MAXL];  // levels >= 1: r_l
  CUtensorMap t[MG_MAXL];  // the up-sweep residual (scratch lin_t with level l's shape)
  CUtensorMap e0;          // level 0's correction, boxed like the iterate (k_update_residual)
  CUtensorMap eh[MG_MAXL]; // the linear up-sweep: e_l with its six-point halo
  CUtensorMap ec[MG_MAXL]; // ... the coarse correction its prolongation reads
  CUtensorMap e0f;         // ... level 0's final correction (scratch lin_wa), boxed like e0
  // the tiled restriction (constant stencils): r_l and e_l of a 32 x 32 tile with the rows
  // and columns the residual needs, and the 16 x 16 coarse tile of r_{l+1}
  CUtensorMap rr0a, rr0b, rr[MG_MAXL], er[MG_MAXL], rc[MG_MAXL];
};
bool build_lin_maps(LinMaps& M, const LevelArrays& A, float* lin_t, float* lin_wa, int nprob, int lstar);

struct CycleArgs {
  ProbDev* probs;
  ProbState* state;
  float* partials;
  int ntiles_max;
  int nprob, n0, L, lstar;
  int nl[MG_MAXL];
  int sk, hk;
  float omega;
  cudaStream_t stream;
  Profiler* prof;
  const int* active;  // device list of the problems cycle launches cover (nullptr: all)
  int nactive;
  const TileMaps* maps;  // host copy of the tensor maps (tiled levels)
  float *xh0, *xl0;      // pitched iterate pair of the tiled path (read by even cycles)
  float *xh0b, *xl0b;    // the second pair (read by odd cycles, written by even ones)
  float *r0a, *r0b;      // the two level-0 residual arrays
  const float* b0;       // pitched level-0 right-hand sides (tiled path)
  bool pdl;              // launch the cycle chain with programmatic dependencies
  int ctail;             // levels >= lstar in one CTA cluster per problem (mg_ctail.cu)
  // HK_LINEAR: scratch vectors of the chain of convolutions and the up-sweep residual,
  // each [nprob][n_l][pitch_l] on the level being processed (sized for level 0)
  float *lin_wa, *lin_wb, *lin_t;
  const LevelArrays* arrays;      // base pointers of the level arrays (host copy)
  const LinMaps* lin_maps;        // tensor maps of the batched level path (host copy)
  int nu1, nu2;                   // smoothing steps; other than 1 only on the batched level path
  int generic;                    // levels above the tail on the batched level path (mg_linear.cu):
                                  // the linear smoother, the kernel stack, or nu other than 1
  int short_wait;                 // test setting copied into the control blocks by launch_bnorm
  int shape;                      // layout of the tiled level kernels (MG_SHAPE_*)
  int strip_rows;                 // MG_SHAPE_PSTRIP: least walk height the strips take
};


// one network evaluation: a stencil field (st) or a constant stencil (s) on an n x n grid
struct NetJob {
  const float* st;
  const float* s;
  float* W;
  int n;
  int pad_;
};

// a uniform batch of stencil fields [nfields][9][n][n] -> kernels [nfields][9][n][n]
struct NetBatch {
  const float* st;
  float* W;
  size_t stride;
  int n;
  int pad_;
};

// Launch with programmatic stream serialisation: the kernel may be scheduled before the
// previous kernel on the stream finishes; it must call griddepcontrol.wait before reading
// anything that kernel writes (all cycle kernels do).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

int tiles_per_side(int n);
size_t tail_smem_bytes(const int* nl, int l0, int L, int hk);

cudaError_t launch_bnorm(const CycleArgs& a, const float* b);
// tiled path (mg_tiles.cu): residual of the pitched iterate with the stopping test, and
// one V-cycle below it ending with the same residual and test for the new iterate
cudaError_t launch_residual(const CycleArgs& a, float rtol, int max_cycles);
// cycle `parity` reads the level-0 residual and the iterate from r[0], (xh0, xl0) (0) or
// r0b, (xh0b, xl0b) (1) and writes the new ones to the other arrays: the fused level-0
// kernel reads both with halos, so it must not overwrite them in place
cudaError_t launch_cycle(const CycleArgs& a, float rtol, int max_cycles, int parity);
bool build_tile_maps(TileMaps& maps, const LevelArrays& arrays, int nprob, int lstar, int shape);
// strip layouts (mg_strip.cu): the r block (box) of the down-sweep, and its launch on level
// l for np problems with the tensor map m of that level's r array
void strip_box(int shape, int* bw, int* bh);
cudaError_t launch_sdown(const CycleArgs& a, const CUtensorMap& m, int l, int np);
// whether the paired strips take level l's down-sweep for np problems (shape MG_SHAPE_PSTRIP;
// the launches they do not take run the 32 x 32 tiles, with bit-identical results)
bool pdown_applies(const CycleArgs& a, int l, int np);
// level 0 after an up-sweep run elsewhere: x += e_0 and the residual of the new iterate
// with the stopping test, on the arrays of cycle `parity` (mg_tiles.cu); e0: tensor map of
// e_0 with the iterate's box (tile_res_box)
cudaError_t launch_update_residual(const CycleArgs& a, const CUtensorMap& e0, float rtol, int max_cycles, int parity);
void tile_res_box(int* bw, int* bh);
// 3-D tensor map {x, y, problem} of a pitched level array, box bw x bh x 1 (mg_tiles.cu)
bool make_map(CUtensorMap* m, float* base, int n, int pitch, int nprob, int bw, int bh);
cudaError_t launch_pack(const float* src, float* dst, int n, int pitch, int nprob, cudaStream_t s);
// dst <- src_a, or src_b for the problems whose count of applied cycles is odd
cudaError_t launch_unpack(const float* src_a, const float* src_b, const ProbState* state, float* dst, int n, int pitch,
                          int nprob, cudaStream_t s);
// coarse tail from level a.lstar: one CTA per problem (mg_cycle.cu), or the cluster tail
// when a.ctail is set; prepare_tail sets launch attributes (call it outside stream capture)
cudaError_t launch_tail(const CycleArgs& a);
cudaError_t prepare_tail(const CycleArgs& a);
// xout[v] = one V-cycle from zero of levels 0 .. L-1 applied to rin[v], v = p * nvec + j
// (dense [nprob * nvec][n0][n0] arrays; contexts whose whole hierarchy runs in one CTA)
cudaError_t launch_tail_vec(const CycleArgs& a, const float* rin, float* xout, int nvec);
// W (9 x n x n per-point kernels) <- its transpose's kernels, through scratch (9 x n x n)
cudaError_t launch_transpose_kernels(float* W, int n, float* scratch, cudaStream_t s);
// the three-kernel stack's fields [27][n][n] <- those of its transpose (blocks reversed, each
// transposed), through scratch (27 x n x n)
cudaError_t launch_transpose_stack(float* W, int n, float* scratch, cudaStream_t s);
bool ctx_tail_args(const ::mg_ctx* ctx, CycleArgs* a);
void ctx_args(const ::mg_ctx* ctx, CycleArgs* a);
cudaError_t launch_tail_solve(const CycleArgs& a, const float* b, float* xhi, float* xlo, float rtol, int max_cycles,
                              int budget, int final_residual);
// cluster tail (mg_ctail.cu): levels lstar .. L-1 in one MG_CT_C-CTA cluster per problem
size_t ctail_smem_bytes(const int* nl, int ls, int L, int hk);
bool ctail_supported(int sk, int hk, size_t smem);
cudaError_t prepare_ctail(const CycleArgs& a);
cudaError_t launch_ctail(const CycleArgs& a);
cudaError_t launch_smoother(const CycleArgs& a, int p, int l, const float* f, float* u, int nsteps);
// t = f - A u of problem p on level l into the level's r vector (dense n_l x n_l)
cudaError_t launch_level_residual(const CycleArgs& a, int p, int l, const float* f, const float* u);
// the batched level path (mg_linear.cu) -- the linear smoother, and nu1, nu2 > 1 with the
// Jacobi or the linear smoother: the cycle's levels above a.lstar in batched level kernels,
// then the one-CTA tail; and the linear smoother's standalone application
cudaError_t launch_cycle_linear(const CycleArgs& a, float rtol, int max_cycles, int parity);
cudaError_t launch_smoother_linear(const CycleArgs& a, int p, int l, const float* f, float* u, int nsteps);
// phi <- the parameters of H^T (chain reversed, kernels mirrored), nlev sets in place
cudaError_t launch_transpose_linear(float* phi, int nlev, cudaStream_t s);

cudaError_t launch_varcoef5(int n, int nprob, const float* cells, size_t cells_stride, float* field,
                            size_t field_stride, cudaStream_t s);
cudaError_t launch_rap_field(ProbDev* probs, int nprob, int l, int nc, cudaStream_t s);
cudaError_t launch_rap_const(ProbDev* probs, int nprob, int L, cudaStream_t s);
cudaError_t launch_coarsest_factor(ProbDev* probs, int nprob, int L, int sk, int* fail, cudaStream_t s);
cudaError_t launch_expand_stencil(const ProbDev* probs, int p, int l, int n, int sk, float* out, cudaStream_t s);
cudaError_t launch_expand_kernels(const ProbDev* probs, int p, int l, int n, int sk, int hk, float omega, float* out,
                                  cudaStream_t s);

cudaError_t launch_net_forward(const NetJob* jobs_dev, int njobs, int nmax, const float* params, float omega, int bf16,
                               cudaStream_t s);
cudaError_t launch_net_forward_batch(const NetBatch& batch, int nfields, const float* params, float omega, int bf16,
                                     cudaStream_t s);
// the three-kernel network (MG_NET_CONV3): [27][n][n] per job, FP32
cudaError_t launch_net_forward3(const NetJob* jobs_dev, int njobs, int nmax, const float* params, float omega,
                                cudaStream_t s);
// the same on a uniform batch (kernels [27][n][n] of field y at batch.W + 3 y batch.stride)
// and its backward (dW laid out like W; partials: net_backward_ctas x MG_NPARAMS_K3)
cudaError_t launch_net_forward3_batch(const NetBatch& batch, int nfields, const float* params, float omega,
                                      cudaStream_t s);
cudaError_t launch_net_backward3(const NetBatch& batch, int nfields, const float* dW, const float* params,
                                 float* partials, float scale, float* grad, cudaStream_t s);
// the shared-kernel network (MG_NET_CONV_SHARED): nsets parameter sets expanded to the dense
// layout (w[o][c] = k_o), and one dense gradient summed back over the input channels
cudaError_t launch_net_expand_shared(const float* shared, float* dense, int nsets, cudaStream_t s);
cudaError_t launch_net_reduce_shared(const float* dense_grad, float* grad, cudaStream_t s);
cudaError_t launch_copy_rel(const ProbState* state, float* rel, int nprob, cudaStream_t s);
int net_backward_ctas(int n, int nfields);
// the fully connected network (mg_netfc.cu); the backward needs fc_backward_floats scratch
cudaError_t launch_fc_forward(const NetJob* jobs_dev, int njobs, int nmax, const float* params, float omega, int bf16,
                              cudaStream_t s);
cudaError_t launch_fc_forward_batch(const NetBatch& batch, int nfields, const float* params, float omega, int bf16,
                                    cudaStream_t s);
// its bfloat16 inference on the tensor cores (mg_fctc.cu): the same jobs and batches
cudaError_t launch_fc_forward_tc(const NetJob* jobs_dev, int njobs, int nmax, const float* params, float omega,
                                 cudaStream_t s);
cudaError_t launch_fc_forward_batch_tc(const NetBatch& batch, int nfields, const float* params, float omega,
                                       cudaStream_t s);
size_t fc_backward_floats(int n, int nfields);
cudaError_t launch_fc_backward(const NetBatch& batch, int nfields, const float* dW, const float* params, int bf16,
                               float* scratch, float scale, float* grad, cudaStream_t s);
cudaError_t launch_net_backward(const NetBatch& batch, int nfields, const float* dW, const float* params, int bf16,
                                float* partials, float scale, float* grad, cudaStream_t s);

// records the thread-local error text of the C ABI and returns `status`
int api_fail(int status, const char* fmt, ...);

}  // namespace mg
