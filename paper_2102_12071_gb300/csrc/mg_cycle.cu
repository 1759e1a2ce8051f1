// mg_cycle.cu -- the V-cycle of Algorithm 1 on the error equation, for sm_103a.
//
// The tiled levels (n_l > MG_TAIL_N) are in mg_tiles.cu.  This file holds
//   k_bnorm      ||b||^2 per problem (float-float) and the reset of the stopping state;
//   k_tail       levels with n_l <= MG_TAIL_N in one CTA per problem, down to the FP64
//                coarsest solve and back up (Algorithm 1, recursion to the coarsest solve and back);
//   k_tail_solve whole solves of small problems (n_0 <= MG_TAIL_N) in one CTA each:
//                compensated residual, stopping test, V-cycle, float-float update;
//   k_level_*    the standalone smoother of mg_smoother_apply.
//
// The cycle on the error equation from e = 0 equals Algorithm 1 applied to x because the
// cycle is linear in (x, b); the outer iterate and residual carry ~48 significand bits.
#include <atomic>

#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_ops.cuh"
#include "mg_reduce.cuh"
#include "mg_tail.cuh"
#include "mg_tma.cuh"

namespace mg {

constexpr int TB = 32;        // fine tile side of the norm kernel
constexpr int NT = 256;       // threads per CTA of the norm kernel
constexpr int TAIL_THREADS = 512;

template <int SK>
__device__ __forceinline__ void load_stencil(const LevelDev& L, float (&s)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
}

// ------------------------------------------------------------------ norms
__global__ void __launch_bounds__(NT) k_bnorm(const ProbDev* __restrict__ probs, ProbState* __restrict__ state,
                                              float* __restrict__ partials, int ntiles_max,
                                              const float* __restrict__ b, int short_wait) {
  const int p = blockIdx.y;
  const int n = probs[p].lv[0].n;
  const size_t nn = (size_t)n * n;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx;
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  const float* bp = b + p * nn;
  float acc = 0.f;
  for (int t = threadIdx.x; t < TB * TB; t += NT) {
    const int i = R0 + t / TB, j = C0 + t % TB;
    if (in_grid(i, j, n)) {
      const float v = bp[(size_t)i * n + j];
      acc = fmaf(v, v, acc);
    }
  }
  float hi, lo;
  if (block_partial_and_last<NT>(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, hi, lo)) {
    if (threadIdx.x == 0) {
      state[p].bb_hi = hi;
      state[p].bb_lo = lo;
      state[p].active = 1;
      state[p].iter = 0;
      state[p].cycles = 0;
      state[p].status = 0;
      state[p].short_wait = short_wait;
      state[p].t_start = global_ns();
    }
  }
}

// ------------------------------------------------------------------ tail
template <int SK, int HK>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail(const ProbDev* __restrict__ probs,
                                                       const ProbState* __restrict__ state, int l0, int L,
                                                       float omega, const int* __restrict__ act) {
  extern __shared__ float sm[];
  __shared__ float sc[MG_MAXL][9];
  __shared__ float wi[MG_MAXL][9];
  __shared__ TailLayout lay;
  pdl_trigger();
  const int p = act ? act[blockIdx.x] : blockIdx.x;
  const ProbDev& P = probs[p];
  if (threadIdx.x == 0) {
    int nl[MG_MAXL];
    for (int l = 0; l < L; ++l) nl[l] = P.lv[l].n;
    tail_layout(nl, l0, L, HK, lay);
  }
  __syncthreads();
  tail_prologue<SK, HK>(P, sm, lay, sc, wi, l0, L);
  pdl_wait();
  if (!st_active(state + p)) return;
  const int n = P.lv[l0].n, m = n + 2, pitch = P.lv[l0].pitch;
  float* r = sm + lay.off_r[l0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  TAIL_FOR(n) r[(i + 1) * m + j + 1] = __ldcg(P.lv[l0].r + (size_t)i * pitch + j);
  __syncthreads();
  tail_cycle<SK, HK>(P, sm, lay, sc, wi, l0, L, omega);
  const float* e = sm + lay.off_e[l0];
  TAIL_FOR(n) P.lv[l0].e[(size_t)i * pitch + j] = e[(i + 1) * m + j + 1];
}

// Whole solves of small problems: up to `budget` iterations of (residual, test, V-cycle,
// update); with `final_residual` one more residual evaluation at the end.
template <int SK, int HK>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_solve(const ProbDev* __restrict__ probs,
                                                             ProbState* __restrict__ state, int L, float omega,
                                                             const float* __restrict__ b, float* __restrict__ xhi,
                                                             float* __restrict__ xlo, float rtol, int max_cycles,
                                                             int budget, int final_residual,
                                                             const int* __restrict__ act) {
  extern __shared__ float sm[];
  __shared__ float sc[MG_MAXL][9];
  __shared__ float wi[MG_MAXL][9];
  __shared__ float wh[TAIL_THREADS / 32], wl[TAIL_THREADS / 32];
  __shared__ TailLayout lay;
  __shared__ int go;
  const int p = act ? act[blockIdx.x] : blockIdx.x;
  if (!st_active(state + p)) return;
  const ProbDev& P = probs[p];
  if (threadIdx.x == 0) {
    int nl[MG_MAXL];
    for (int l = 0; l < L; ++l) nl[l] = P.lv[l].n;
    tail_layout(nl, 0, L, HK, lay);
  }
  __syncthreads();
  tail_prologue<SK, HK>(P, sm, lay, sc, wi, 0, L);
  const LevelDev& L0 = P.lv[0];
  const int n = L0.n, m = n + 2;
  const size_t nn = (size_t)n * n;
  const float* bp = b + p * nn;
  float* xh = xhi + p * nn;
  float* xl = xlo ? xlo + p * nn : nullptr;
  float* r = sm + lay.off_r[0];
  const float* e = sm + lay.off_e[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __syncthreads();
  for (int it = 0; it <= budget; ++it) {
    if (it == budget && !final_residual) break;
    // residual of the current iterate (compensated), its norm and the stopping test
    float acc = 0.f;
    TAIL_FOR(n) {
      const int q = i * n + j;
      float hi = bp[q], lo = 0.f;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
        if (!in_grid(ii, jj, n)) continue;
        const float a = (SK == SK_CONST) ? sc[0][k] : __ldg(L0.st + k * nn + q);
        const float x = xh[ii * n + jj];
        const float pr = __fmul_rn(a, x), pe = fmaf(a, x, -pr);
        float sum, err;
        two_sum(hi, -pr, sum, err);
        hi = sum;
        lo += err - pe;
        if (xl) lo = fmaf(-a, xl[ii * n + jj], lo);
      }
      const float rv = hi + lo;
      r[(i + 1) * m + j + 1] = rv;
      acc = fmaf(rv, rv, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      wh[warp] = acc;
      wl[warp] = 0.f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float hi = 0.f, lo = 0.f;
      for (int k = 0; k < nwarps; ++k) ff_add(hi, lo, wh[k], wl[k]);
      decide(state[p], hi, lo, rtol, max_cycles);
      go = st_active(state + p) && it < budget;
    }
    __syncthreads();
    if (!go) break;
    tail_cycle<SK, HK>(P, sm, lay, sc, wi, 0, L, omega);
    // x += e_0 (float-float)
    TAIL_FOR(n) {
      const int q = i * n + j;
      const float ev = e[(i + 1) * m + j + 1];
      if (xl) {
        float hi = xh[q], lo = xl[q], sum, err;
        two_sum(hi, ev, sum, err);
        err += lo;
        fast_two_sum(sum, err, hi, lo);
        xh[q] = hi;
        xl[q] = lo;
      } else {
        xh[q] += ev;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- standalone smoother
// t = f - A u into the level's r vector (dense scratch, one thread per point)
template <int SK>
__global__ void k_level_residual(const ProbDev* __restrict__ probs, int p, int l, const float* __restrict__ f,
                                 const float* __restrict__ u) {
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  float s[9];
  load_stencil<SK>(L, s);
  const int i = q / n, j = q % n;
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
    const float a = (SK == SK_CONST) ? s[k] : L.st[(size_t)k * n * n + q];
    acc = fmaf(a, in_grid(ii, jj, n) ? u[ii * n + jj] : 0.f, acc);
  }
  L.r[q] = f[q] - acc;
}

// u += H t with t the level's r vector
template <int SK, int HK>
__global__ void k_level_smooth(const ProbDev* __restrict__ probs, int p, int l, float omega, float* __restrict__ u) {
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  float s[9];
  load_stencil<SK>(L, s);
  const int i = q / n, j = q % n;
  const float* t = L.r;
  if (HK == HK_JACOBI) {
    const float d = (SK == SK_CONST) ? s[4] : L.st[4 * (size_t)n * n + q];
    u[q] += (omega / d) * t[q];
    return;
  }
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
    float w;
    if (HK == HK_TABLE) w = L.W[k * L.T * L.T + kclass(i, n, L.T) * L.T + kclass(j, n, L.T)];
    else w = L.W[(size_t)k * n * n + q];
    acc = fmaf(w, in_grid(ii, jj, n) ? t[ii * n + jj] : 0.f, acc);
  }
  u[q] += acc;
}

// ---------------------------------------------------------------- launchers
int tiles_per_side(int n) { return (n + TB - 1) / TB; }

cudaError_t launch_bnorm(const CycleArgs& a, const float* b) {
  const int nt = tiles_per_side(a.n0);
  dim3 grid(nt * nt, a.nprob);
  a.prof->launches++;
  // norm partial slots start empty (see block_partial_and_last)
  cudaError_t e = cudaMemsetAsync(a.partials, 0xff, sizeof(float) * (size_t)a.nprob * a.ntiles_max, a.stream);
  if (e != cudaSuccess) return e;
  k_bnorm<<<grid, NT, 0, a.stream>>>(a.probs, a.state, a.partials, a.ntiles_max, b, a.short_wait);
  return cudaGetLastError();
}

static inline int nlaunch(const CycleArgs& a) { return (a.active && a.nactive > 0) ? a.nactive : a.nprob; }

size_t tail_smem_bytes(const int* nl, int l0, int L, int hk) {
  TailLayout lay;
  tail_layout(nl, l0, L, hk, lay);
  return (size_t)lay.total * sizeof(float);
}

// The tail kernels need more than the default 48 KB of dynamic shared memory; the limit is
// raised once per device to the largest layout any context may use (MG_TAIL_SMEM_MAX).
template <int SK, int HK>
static cudaError_t set_tail_attrs(size_t smem) {
  static std::atomic<int> done[64];
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(k_tail<SK, HK>, cudaFuncAttributeMaxDynamicSharedMemorySize, MG_TAIL_SMEM_MAX);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tail_solve<SK, HK>, cudaFuncAttributeMaxDynamicSharedMemorySize, MG_TAIL_SMEM_MAX);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev].store(1, std::memory_order_release);
  return e;
}

cudaError_t prepare_tail(const CycleArgs& a) {
  if (a.ctail) return prepare_ctail(a);
  const size_t smem = tail_smem_bytes(a.nl, a.lstar, a.L, a.hk);
  cudaError_t e;
  MG_DISPATCH_T(a.sk, a.hk, (e = set_tail_attrs<SK_, HK_>(smem)));
  return e;
}

cudaError_t launch_tail(const CycleArgs& a) {
  if (a.ctail) return launch_ctail(a);
  const int ls = a.lstar, L = a.L;
  const size_t smem = tail_smem_bytes(a.nl, ls, L, a.hk);
  cudaError_t e;
  MG_DISPATCH_T(a.sk, a.hk, (e = set_tail_attrs<SK_, HK_>(smem)));
  if (e != cudaSuccess) return e;
  a.prof->launches++;
  a.prof->begin(PK_TAIL, a.stream);
  const ProbDev* probs = a.probs;
  const ProbState* state = a.state;
  MG_DISPATCH_T(a.sk, a.hk, (e = launch_pdl(a.pdl, k_tail<SK_, HK_>, dim3(nlaunch(a)), dim3(TAIL_THREADS), smem,
                                          a.stream, probs, state, ls, L, a.omega, a.active)));
  a.prof->end(a.stream);
  return e;
}

cudaError_t launch_tail_solve(const CycleArgs& a, const float* b, float* xhi, float* xlo, float rtol, int max_cycles,
                              int budget, int final_residual) {
  const size_t smem = tail_smem_bytes(a.nl, 0, a.L, a.hk);
  cudaError_t e;
  MG_DISPATCH_T(a.sk, a.hk, (e = set_tail_attrs<SK_, HK_>(smem)));
  if (e != cudaSuccess) return e;
  a.prof->launches++;
  a.prof->begin(PK_TAIL, a.stream);
  MG_DISPATCH_T(a.sk, a.hk, (k_tail_solve<SK_, HK_><<<nlaunch(a), TAIL_THREADS, smem, a.stream>>>(
                              a.probs, a.state, a.L, a.omega, b, xhi, xlo, rtol, max_cycles, budget, final_residual,
                              a.active)));
  a.prof->end(a.stream);
  return cudaGetLastError();
}

// One V-cycle from zero of levels 0 .. L-1 on nvec right-hand sides per problem: the
// coarse solve of Algorithm 2's training objective (one CTA per vector, every level in
// shared memory).  rin, xout: dense [nprob * nvec][n0][n0].
template <int SK, int HK>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_vec(const ProbDev* __restrict__ probs, int L, float omega,
                                                           const float* __restrict__ rin, float* __restrict__ xout,
                                                           int nvec) {
  extern __shared__ float sm[];
  __shared__ float sc[MG_MAXL][9];
  __shared__ float wi[MG_MAXL][9];
  __shared__ TailLayout lay;
  const int v = blockIdx.x, p = v / nvec;
  const ProbDev& P = probs[p];
  if (threadIdx.x == 0) {
    int nl[MG_MAXL];
    for (int l = 0; l < L; ++l) nl[l] = P.lv[l].n;
    tail_layout(nl, 0, L, HK, lay);
  }
  __syncthreads();
  tail_prologue<SK, HK>(P, sm, lay, sc, wi, 0, L);
  const int n = P.lv[0].n, m = n + 2;
  const size_t nn = (size_t)n * n;
  const float* src = rin + (size_t)v * nn;
  float* r = sm + lay.off_r[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  TAIL_FOR(n) r[(i + 1) * m + j + 1] = src[(size_t)i * n + j];
  __syncthreads();
  tail_cycle<SK, HK>(P, sm, lay, sc, wi, 0, L, omega);
  const float* e = sm + lay.off_e[0];
  float* dst = xout + (size_t)v * nn;
  TAIL_FOR(n) dst[(size_t)i * n + j] = e[(i + 1) * m + j + 1];
}

cudaError_t launch_tail_vec(const CycleArgs& a, const float* rin, float* xout, int nvec) {
  const size_t smem = tail_smem_bytes(a.nl, 0, a.L, a.hk);
  cudaError_t e;
  MG_DISPATCH_T(a.sk, a.hk, (e = set_tail_attrs<SK_, HK_>(smem)));
  if (e != cudaSuccess) return e;
  MG_DISPATCH_T(a.sk, a.hk, (k_tail_vec<SK_, HK_><<<a.nprob * nvec, TAIL_THREADS, smem, a.stream>>>(
                              a.probs, a.L, a.omega, rin, xout, nvec)));
  return cudaGetLastError();
}

// out[k][y] = W[8 - k][y + d_k] (zero outside): the kernels of H^T
__global__ void k_transpose_kernels(const float* __restrict__ W, float* __restrict__ out, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 9 * n * n) return;
  const int k = q / (n * n), y = q % (n * n), i = y / n, j = y % n;
  const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
  out[q] = in_grid(ii, jj, n) ? W[(size_t)(8 - k) * n * n + ii * n + jj] : 0.f;
}

cudaError_t launch_transpose_kernels(float* W, int n, float* scratch, cudaStream_t s) {
  const int cnt = 9 * n * n;
  k_transpose_kernels<<<(cnt + 255) / 256, 256, 0, s>>>(W, scratch, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(W, scratch, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, s);
}

// The kernels of the stack H = K3 K2 K1 transposed: H^T = K1^T K2^T K3^T, stored in the
// order the stack is applied (first block first), so out = (K3^T, K2^T, K1^T) with each
// block transposed as above; W holds the three blocks [27][n][n].
__global__ void k_transpose_stack(const float* __restrict__ W, float* __restrict__ out, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = n * n;
  if (q >= 27 * nn) return;
  const int b = q / (9 * nn), r = q % (9 * nn), k = r / nn, y = r % nn, i = y / n, j = y % n;
  const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
  out[q] = in_grid(ii, jj, n) ? W[(size_t)(2 - b) * 9 * nn + (size_t)(8 - k) * nn + ii * n + jj] : 0.f;
}

cudaError_t launch_transpose_stack(float* W, int n, float* scratch, cudaStream_t s) {
  const int cnt = 27 * n * n;
  k_transpose_stack<<<(cnt + 255) / 256, 256, 0, s>>>(W, scratch, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(W, scratch, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, s);
}

cudaError_t launch_level_residual(const CycleArgs& a, int p, int l, const float* f, const float* u) {
  const int n = a.nl[l];
  const int nb = (n * n + 255) / 256;
  a.prof->launches++;
  if (a.sk == SK_CONST) k_level_residual<SK_CONST><<<nb, 256, 0, a.stream>>>(a.probs, p, l, f, u);
  else k_level_residual<SK_FIELD><<<nb, 256, 0, a.stream>>>(a.probs, p, l, f, u);
  return cudaGetLastError();
}

cudaError_t launch_smoother(const CycleArgs& a, int p, int l, const float* f, float* u, int nsteps) {
  if (a.hk == HK_LINEAR) return launch_smoother_linear(a, p, l, f, u, nsteps);
  if (a.hk == HK_STACK3) return cudaErrorNotSupported;  // refused by mg_smoother_apply
  const int n = a.nl[l];
  const int nb = (n * n + 255) / 256;
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = launch_level_residual(a, p, l, f, u);
    if (e != cudaSuccess) return e;
    a.prof->launches++;
    MG_DISPATCH(a.sk, a.hk, (k_level_smooth<SK_, HK_><<<nb, 256, 0, a.stream>>>(a.probs, p, l, a.omega, u)));
  }
  return cudaGetLastError();
}

__global__ void k_copy_rel(const ProbState* __restrict__ state, float* __restrict__ rel, int nprob) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nprob) rel[p] = state[p].rel;
}

cudaError_t launch_copy_rel(const ProbState* state, float* rel, int nprob, cudaStream_t s) {
  k_copy_rel<<<(nprob + 127) / 128, 128, 0, s>>>(state, rel, nprob);
  return cudaGetLastError();
}

}  // namespace mg
