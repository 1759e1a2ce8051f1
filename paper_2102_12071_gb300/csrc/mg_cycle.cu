// mg_cycle.cu -- the V-cycle of Algorithm 1 on the error equation, for sm_103a.
//
// The tiled levels (n_l > MG_TAIL_N) are in mg_tiles.cu.  This file holds
//   k_bnorm      ||b||^2 per problem (float-float) and the reset of the stopping state;
//   k_tail       levels with n_l <= MG_TAIL_N in one CTA per problem, down to the FP64
//                coarsest solve and back up (Algorithm 1 lines 3-9);
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
#include "mg_tma.cuh"

namespace mg {

constexpr int TB = 32;        // fine tile side of k_residual / k_down / k_up
constexpr int NT = 256;       // threads per CTA of the tiled kernels
constexpr int TAIL_THREADS = 512;

template <int SK>
__device__ __forceinline__ void load_stencil(const LevelDev& L, float (&s)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
}

// ------------------------------------------------------------------ norms
__global__ void __launch_bounds__(NT) k_bnorm(const ProbDev* __restrict__ probs, ProbState* __restrict__ state,
                                              float* __restrict__ partials, int ntiles_max,
                                              const float* __restrict__ b) {
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
    if (in_grid(i, j, n)) { const float v = bp[(size_t)i * n + j]; acc = fmaf(v, v, acc); }
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
    }
  }
}

// ------------------------------------------------------------------ tail
// Levels l0 .. L-1 of one problem in one CTA with every vector in shared memory.
struct TailLayout {
  int off_r[MG_MAXL], off_e[MG_MAXL], off_w[MG_MAXL];
  int off_t, total;
};

__host__ __device__ inline void tail_layout(const int* nl, int l0, int L, int hk, TailLayout& t) {
  int o = 0;
  for (int l = l0; l < L; ++l) {
    t.off_r[l] = o; o += nl[l] * nl[l];
    t.off_e[l] = o; o += nl[l] * nl[l];
  }
  t.off_t = o; o += nl[l0] * nl[l0];
  for (int l = l0; l < L; ++l) {
    t.off_w[l] = o;
    if (hk == HK_TABLE && l < L - 1) {
      const int T = nl[l] < MG_PROXY ? nl[l] : MG_PROXY;
      o += 9 * T * T;
    }
  }
  t.total = o;
}

template <int SK>
__device__ __forceinline__ float tail_A(const LevelDev& L, const float* s, const float* v, int n, int i, int j) {
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
    const float a = (SK == SK_CONST) ? s[k] : __ldg(L.st + (size_t)k * n * n + (size_t)i * n + j);
    const float x = in_grid(ii, jj, n) ? v[ii * n + jj] : 0.f;
    acc = (k == 0) ? a * x : fmaf(a, x, acc);
  }
  return acc;
}

template <int SK, int HK>
__device__ __forceinline__ float tail_H(const LevelDev& L, const float* s, const float* wtab, float omega,
                                        const float* v, int n, int i, int j) {
  if (HK == HK_JACOBI) {
    const float d = (SK == SK_CONST) ? s[4] : __ldg(L.st + 4 * (size_t)n * n + (size_t)i * n + j);
    return omega * v[i * n + j] / d;
  }
  const float* w;
  int stride;
  if (HK == HK_TABLE) {
    const int T = L.T;
    w = wtab + kclass(i, n, T) * T + kclass(j, n, T);
    stride = T * T;
  } else {
    w = L.W + (size_t)i * n + j;
    stride = n * n;
  }
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
    const float x = in_grid(ii, jj, n) ? v[ii * n + jj] : 0.f;
    acc = fmaf(w[k * stride], x, acc);
  }
  return acc;
}

// Down and up sweeps from level l0 with r_{l0} already in shared memory; leaves e_{l0}.
// Loops run warp-per-row, lane-per-column (no integer division); the coarsest level is one
// FP64 product with the precomputed inverse of A_L (one thread per unknown).
#define TAIL_FOR(nside) \
  for (int i = warp; i < (nside); i += nwarps) \
    for (int j = lane; j < (nside); j += 32)

template <int SK, int HK>
__device__ void tail_cycle(const ProbDev& P, float* sm, const TailLayout& lay, const float (*sc)[9], int l0,
                           int L, float omega) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int l = l0; l < L - 1; ++l) {
    const LevelDev& Lv = P.lv[l];
    const int n = Lv.n, nc = P.lv[l + 1].n;
    float* r = sm + lay.off_r[l];
    float* e = sm + lay.off_e[l];
    float* t = sm + lay.off_t;
    const float* w = sm + lay.off_w[l];
    TAIL_FOR(n) e[i * n + j] = tail_H<SK, HK>(Lv, sc[l], w, omega, r, n, i, j);
    __syncthreads();
    TAIL_FOR(n) t[i * n + j] = r[i * n + j] - tail_A<SK>(Lv, sc[l], e, n, i, j);
    __syncthreads();
    float* rc = sm + lay.off_r[l + 1];
    for (int I = warp; I < nc; I += nwarps)
      for (int J = lane; J < nc; J += 32) rc[I * nc + J] = restrict_at(t + (2 * I + 1) * n + 2 * J + 1, n);
    __syncthreads();
  }
  {
    const float* r = sm + lay.off_r[L - 1];
    float* e = sm + lay.off_e[L - 1];
    const int m = P.m;
    if ((int)threadIdx.x < m) {
      const double* Ai = P.chol + threadIdx.x * m;
      double acc = 0.0;
      for (int k = 0; k < m; ++k) acc = fma(Ai[k], (double)r[k], acc);
      e[threadIdx.x] = (float)acc;
    }
    __syncthreads();
  }
  for (int l = L - 2; l >= l0; --l) {
    const LevelDev& Lv = P.lv[l];
    const int n = Lv.n, nc = P.lv[l + 1].n;
    float* r = sm + lay.off_r[l];
    float* e = sm + lay.off_e[l];
    float* t = sm + lay.off_t;
    const float* ec = sm + lay.off_e[l + 1];
    const float* w = sm + lay.off_w[l];
    TAIL_FOR(n) {
      float v = 0.f;
      for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
          const int fi = i + di, fj = j + dj;  // candidate coarse centre 2I+1
          if ((fi & 1) && (fj & 1)) {
            const int I = (fi - 1) >> 1, J = (fj - 1) >> 1;
            if (in_grid(I, J, nc)) v += (di ? 0.5f : 1.f) * (dj ? 0.5f : 1.f) * ec[I * nc + J];
          }
        }
      e[i * n + j] += v;
    }
    __syncthreads();
    TAIL_FOR(n) t[i * n + j] = r[i * n + j] - tail_A<SK>(Lv, sc[l], e, n, i, j);
    __syncthreads();
    TAIL_FOR(n) e[i * n + j] += tail_H<SK, HK>(Lv, sc[l], w, omega, t, n, i, j);
    __syncthreads();
  }
}

template <int SK, int HK>
__device__ void tail_prologue(const ProbDev& P, float* sm, const TailLayout& lay, float (*sc)[9], int l0, int L) {
  for (int l = l0; l < L; ++l) {
    if (SK == SK_CONST && threadIdx.x < 9) sc[l][threadIdx.x] = P.lv[l].s[threadIdx.x];
    if (HK == HK_TABLE && l < L - 1) {
      const int cnt = 9 * P.lv[l].T * P.lv[l].T;
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) sm[lay.off_w[l] + t] = P.lv[l].W[t];
    }
  }
}

template <int SK, int HK>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail(const ProbDev* __restrict__ probs,
                                                       const ProbState* __restrict__ state, int l0, int L,
                                                       float omega, const int* __restrict__ act) {
  extern __shared__ float sm[];
  __shared__ float sc[MG_MAXL][9];
  pdl_trigger();
  const int p = act ? act[blockIdx.x] : blockIdx.x;
  const ProbDev& P = probs[p];
  __shared__ TailLayout lay;
  if (threadIdx.x == 0) {
    int nl[MG_MAXL];
    for (int l = 0; l < L; ++l) nl[l] = P.lv[l].n;
    tail_layout(nl, l0, L, HK, lay);
  }
  __syncthreads();
  tail_prologue<SK, HK>(P, sm, lay, sc, l0, L);
  pdl_wait();
  if (!state[p].active) return;
  const int n = P.lv[l0].n;
  float* r = sm + lay.off_r[l0];
  const int pitch = P.lv[l0].pitch;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) r[q] = P.lv[l0].r[(q / n) * pitch + q % n];
  __syncthreads();
  tail_cycle<SK, HK>(P, sm, lay, sc, l0, L, omega);
  const float* e = sm + lay.off_e[l0];
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) P.lv[l0].e[(q / n) * pitch + q % n] = e[q];
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
  __shared__ float wh[TAIL_THREADS / 32], wl[TAIL_THREADS / 32];
  __shared__ int go;
  const int p = act ? act[blockIdx.x] : blockIdx.x;
  if (!state[p].active) return;
  const ProbDev& P = probs[p];
  __shared__ TailLayout lay;
  if (threadIdx.x == 0) {
    int nl[MG_MAXL];
    for (int l = 0; l < L; ++l) nl[l] = P.lv[l].n;
    tail_layout(nl, 0, L, HK, lay);
  }
  __syncthreads();
  tail_prologue<SK, HK>(P, sm, lay, sc, 0, L);
  const LevelDev& L0 = P.lv[0];
  const int n = L0.n;
  const size_t nn = (size_t)n * n;
  const float* bp = b + p * nn;
  float* xh = xhi + p * nn;
  float* xl = xlo ? xlo + p * nn : nullptr;
  float* r = sm + lay.off_r[0];
  const float* e = sm + lay.off_e[0];
  __syncthreads();
  for (int it = 0; it <= budget; ++it) {
    if (it == budget && !final_residual) break;
    // residual of the current iterate (compensated), its norm and the stopping test
    float acc = 0.f;
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
      const int i = q / n, j = q % n;
      float hi = bp[q], lo = 0.f;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
        if (!in_grid(ii, jj, n)) continue;
        const float a = (SK == SK_CONST) ? sc[0][k] : __ldg(L0.st + k * nn + q);
        const float x = xh[ii * n + jj];
        const float pr = a * x, pe = fmaf(a, x, -pr);
        float sum, err;
        two_sum(hi, -pr, sum, err);
        hi = sum;
        lo += err - pe;
        if (xl) lo = fmaf(-a, xl[ii * n + jj], lo);
      }
      const float rv = hi + lo;
      r[q] = rv;
      acc = fmaf(rv, rv, acc);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) { wh[threadIdx.x >> 5] = acc; wl[threadIdx.x >> 5] = 0.f; }
    __syncthreads();
    if (threadIdx.x == 0) {
      float hi = 0.f, lo = 0.f;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) ff_add(hi, lo, wh[k], wl[k]);
      decide(state[p], hi, lo, rtol, max_cycles);
      go = state[p].active && it < budget;
    }
    __syncthreads();
    if (!go) break;
    tail_cycle<SK, HK>(P, sm, lay, sc, 0, L, omega);
    // x += e_0 (float-float)
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
      if (xl) {
        float hi = xh[q], lo = xl[q], sum, err;
        two_sum(hi, e[q], sum, err);
        err += lo;
        fast_two_sum(sum, err, hi, lo);
        xh[q] = hi;
        xl[q] = lo;
      } else {
        xh[q] += e[q];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- standalone smoother
// t = f - A u into the level's r vector (one thread per point)
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
  u[q] += tail_H<SK, HK>(L, s, L.W, omega, L.r, n, q / n, q % n);
}

// ---------------------------------------------------------------- launchers
int tiles_per_side(int n) { return (n + TB - 1) / TB; }

cudaError_t launch_bnorm(const CycleArgs& a, const float* b) {
  const int nt = tiles_per_side(a.n0);
  dim3 grid(nt * nt, a.nprob);
  a.prof->launches++;
  k_bnorm<<<grid, NT, 0, a.stream>>>(a.probs, a.state, a.partials, a.ntiles_max, b);
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
  const size_t smem = tail_smem_bytes(a.nl, a.lstar, a.L, a.hk);
  cudaError_t e;
  MG_DISPATCH(a.sk, a.hk, (e = set_tail_attrs<SK_, HK_>(smem)));
  return e;
}

cudaError_t launch_tail(const CycleArgs& a) {
  const int ls = a.lstar, L = a.L;
  const size_t smem = tail_smem_bytes(a.nl, ls, L, a.hk);
  cudaError_t e;
  MG_DISPATCH(a.sk, a.hk, (e = set_tail_attrs<SK_, HK_>(smem)));
  if (e != cudaSuccess) return e;
  a.prof->launches++;
  a.prof->begin(PK_TAIL, a.stream);
  const ProbDev* probs = a.probs;
  const ProbState* state = a.state;
  MG_DISPATCH(a.sk, a.hk, (e = launch_pdl(a.pdl, k_tail<SK_, HK_>, dim3(nlaunch(a)), dim3(TAIL_THREADS), smem, a.stream,
                                          probs, state, ls, L, a.omega, a.active)));
  a.prof->end(a.stream);
  return e;
}

cudaError_t launch_tail_solve(const CycleArgs& a, const float* b, float* xhi, float* xlo, float rtol, int max_cycles,
                              int budget, int final_residual) {
  const size_t smem = tail_smem_bytes(a.nl, 0, a.L, a.hk);
  cudaError_t e;
  MG_DISPATCH(a.sk, a.hk, (e = set_tail_attrs<SK_, HK_>(smem)));
  if (e != cudaSuccess) return e;
  a.prof->launches++;
  a.prof->begin(PK_TAIL, a.stream);
  MG_DISPATCH(a.sk, a.hk, (k_tail_solve<SK_, HK_><<<nlaunch(a), TAIL_THREADS, smem, a.stream>>>(
                              a.probs, a.state, a.L, a.omega, b, xhi, xlo, rtol, max_cycles, budget, final_residual,
                              a.active)));
  a.prof->end(a.stream);
  return cudaGetLastError();
}

cudaError_t launch_smoother(const CycleArgs& a, int p, int l, const float* f, float* u, int nsteps) {
  const int n = a.nl[l];
  const int nb = (n * n + 255) / 256;
  for (int s = 0; s < nsteps; ++s) {
    a.prof->launches += 2;
    if (a.sk == SK_CONST) k_level_residual<SK_CONST><<<nb, 256, 0, a.stream>>>(a.probs, p, l, f, u);
    else k_level_residual<SK_FIELD><<<nb, 256, 0, a.stream>>>(a.probs, p, l, f, u);
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
