// mg_tiles.cu -- the tiled level kernels of the batched V-cycle (the levels above the
// coarse tail).
//
// Each CTA owns a 32 x 32 block of fine points of one problem.  All its inputs, halos
// included, arrive as TMA bulk tensor copies issued by one thread into shared memory
// (one mbarrier per CTA); the copy engine zero-fills everything outside the grid, which is
// exactly the homogeneous Dirichlet exterior.  Level vectors use a row pitch that is a
// multiple of 32 floats (128-byte rows) and all problems of a level are one 3-D tensor
// {x, y, problem}, so one tensor map serves the whole batch.  Threads walk vertical strips
// of a region with the 3x3 neighbourhood in registers (three shared-memory loads per
// point); tiles away from the edges skip all masking, and k_down writes its outputs back
// with TMA stores.
//   k_residual  r = b - A (x_hi + x_lo), compensated (float-float), ||r||^2, stopping test
//   k_down(l)   e = H r, s = r - A e, r_{l+1} = P^T s         (Algorithm 1, pre-smoothing and restriction)
//   k_up(l)     e1 = e + P e_{l+1}, e = e1 + H (r - A e1)      (Algorithm 1, correction and post-smoothing);
//               on level 0 (k_up0) the correction is added to the float-float iterate and the
//               next residual and stopping test follow in the same kernel; k_up0p does the
//               same on constant stencils with two columns per thread in packed FP32.
//   k_update_residual  x += e_0 and the compensated residual with the stopping test, for
//               cycles whose up-sweep ran in the batched level kernels (mg_linear.cu).
#include <cudaTypedefs.h>

#include <atomic>

#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_ops.cuh"
#include "mg_pair.cuh"
#include "mg_reduce.cuh"
#include "mg_tile.cuh"
#include "mg_tma.cuh"

namespace mg {

constexpr int TB = 32;           // fine tile side
constexpr int NT = 256;          // threads per CTA (8 warps)
constexpr int NW = NT / 32;
constexpr int TC = TB / 2;       // coarse tile side
constexpr int XW = TB + 8;       // box width: columns C0-4 .. C0+35 (x start 16-byte aligned)
constexpr int RES_H = TB + 2;    // k_residual x boxes: rows R0-1 .. R0+32
constexpr int DN_H = TB + 5;     // k_down r box: rows R0-2 .. R0+34
constexpr int UPE_H = TB + 4;    // k_up e box: rows R0-2 .. R0+33
constexpr int UPR_H = TB + 2;    // k_up r box: rows R0-1 .. R0+32
constexpr int EC_W = TB / 2 + 8; // k_up coarse box: columns C0/2-4 .. C0/2+19
constexpr int EC_H = TB / 2 + 3; //                  rows    R0/2-2 .. R0/2+16
constexpr int ES = TB + 3;       // k_down e buffer side (rows/cols R0-1 .. R0+33)
// Row stride of that buffer.  The residual pass reads it in 5-row strips of 33 columns, so
// a warp spans two strips; 5 * 45 = 1 (mod 32) puts the second strip's lanes exactly on
// the banks the first strip's lanes leave free (a stride of 35 made most loads 2-way).
constexpr int ESP = 45;
constexpr int UP0E_H = TB + 6;   // k_up0 e box: rows R0-3 .. R0+34
constexpr int UP0R_H = TB + 4;   // k_up0 r box: rows R0-2 .. R0+33
constexpr int EC0_H = TB / 2 + 4; // k_up0 coarse box: rows R0/2-2 .. R0/2+17
// Constant-stencil kernels are bounded to 8 CTAs of 256 threads per SM (32 registers): the
// tile kernels wait ~2.5 us for each tile's copies and more resident CTAs hide more of it.
// The per-point-field variants hold more state and would spill at that bound; their
// bounds (6 CTAs, 4 for k_up0) give the register counts they reach without spilling.
// a tile is "inner" when every point its kernels evaluate lies inside the grid and at
// least MG_NET_MARGIN from the edges: no masking, interior network kernel in registers
constexpr int INNER = 8;

__device__ __forceinline__ bool inner_tile(int R0, int C0, int n) {
  return R0 >= INNER && C0 >= INNER && R0 + TB + INNER <= n && C0 + TB + INNER <= n;
}

// A v at grid point (i, j)
template <int SK>
__device__ __forceinline__ float tapply_A(const LevelDev& L, const float (&s)[9], int i, int j, const Win& v) {
  if (SK == SK_CONST) return dot9(s, v);
  const size_t nn = (size_t)L.n * L.n;
  const float* a = L.st + (size_t)i * L.n + j;
  float w[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = __ldg(a + k * nn);
  return dot9(w, v);
}

// H v at grid point (i, j).  Jacobi: (omega / D) v; table: the interior kernel wi on inner
// tiles, else the point's class from the shared-memory table; field: per-point kernels.
template <int SK, int HK, bool IN>
__device__ __forceinline__ float tapply_H(const LevelDev& L, const float (&s)[9], const float* wtab,
                                          const float (&wi)[9], float omega, int i, int j, const Win& v) {
  if (HK == HK_JACOBI) {
    const float d = (SK == SK_CONST) ? s[4] : __ldg(L.st + 4 * (size_t)L.n * L.n + (size_t)i * L.n + j);
    return (omega / d) * v.b1;
  }
  if (HK == HK_TABLE && IN) return dot9(wi, v);
  float w[9];
  if (HK == HK_TABLE) {
    const int T = L.T;
    const float* p = wtab + kclass(i, L.n, T) * T + kclass(j, L.n, T);
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = p[k * T * T];
  } else {
    const size_t nn = (size_t)L.n * L.n;
    const float* p = L.W + (size_t)i * L.n + j;
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = __ldg(p + k * nn);
  }
  return dot9(w, v);
}

// Network kernels of a constant-stencil level for one tile: the interior kernel to
// registers on inner tiles, else the whole class table to shared memory.
__device__ __forceinline__ void load_table(const LevelDev& L, bool in, float* wtab, float (&wi)[9]) {
  const int T = L.T, M = MG_NET_MARGIN;
  if (in) {
#pragma unroll
    for (int k = 0; k < 9; ++k) wi[k] = L.W[k * T * T + M * T + M];
  } else {
    const int cnt = 9 * T * T;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) wtab[t] = L.W[t];
  }
}

__device__ __forceinline__ bool inside(int i, int j, int n) { return (unsigned)i < (unsigned)n && (unsigned)j < (unsigned)n; }

// ------------------------------------------------------------------ k_residual
// Thread = column of the tile (lane) x strip of 4 rows (warp); 3x3 windows of x_hi and x_lo
// slide down the strip in registers.
// With xo_hi/xo_lo (level-0 pitched arrays of problem p) it also stores the iterate of
// the owned points.
template <int SK, bool IN>
__device__ __forceinline__ float residual_tile(const LevelDev& L, const float (&s)[9], const float* XH,
                                               const float* XL, const float* BB, int R0, int C0, float* rdst,
                                               float* xo_hi = nullptr, float* xo_lo = nullptr,
                                               const float* bg = nullptr) {
  constexpr int KS = TB / NW;
  const int n = L.n, pitch = L.pitch;
  const int tj = threadIdx.x & 31, t0 = (threadIdx.x >> 5) * KS, j = C0 + tj;
  const float* ch = XH + (t0 + 1) * XW + tj + 4;
  const float* cl = XL + (t0 + 1) * XW + tj + 4;
  Win h, l;
  h.load_ab(ch, XW);
  l.load_ab(cl, XW);
  float acc = 0.f;
  const size_t g0 = (size_t)(R0 + t0) * pitch + j;
  float* rout = rdst + g0;
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    h.load_c(ch + k * XW, XW);
    l.load_c(cl + k * XW, XW);
    const int i = R0 + t0 + k;
    if (IN || inside(i, j, n)) {
      float a[9];
      if (SK == SK_CONST) {
#pragma unroll
        for (int q = 0; q < 9; ++q) a[q] = s[q];
      } else {
        const size_t nn = (size_t)n * n;
        const float* ap = L.st + (size_t)i * n + j;
#pragma unroll
        for (int q = 0; q < 9; ++q) a[q] = __ldg(ap + q * nn);
      }
      // b: the tile in shared memory, or (bg, the problem's pitched array) one coalesced
      // global load per point
      float hi = bg ? __ldg(bg + g0 + (size_t)k * pitch) : BB[(t0 + k) * TB + tj], lo = 0.f;
      dot2_sub(a[0], h.a0, l.a0, hi, lo);
      dot2_sub(a[1], h.a1, l.a1, hi, lo);
      dot2_sub(a[2], h.a2, l.a2, hi, lo);
      dot2_sub(a[3], h.b0, l.b0, hi, lo);
      dot2_sub(a[4], h.b1, l.b1, hi, lo);
      dot2_sub(a[5], h.b2, l.b2, hi, lo);
      dot2_sub(a[6], h.c0, l.c0, hi, lo);
      dot2_sub(a[7], h.c1, l.c1, hi, lo);
      dot2_sub(a[8], h.c2, l.c2, hi, lo);
      const float r = hi + lo;
      rout[k * pitch] = r;
      acc = fmaf(r, r, acc);
      if (xo_hi) {
        xo_hi[g0 + (size_t)k * pitch] = h.b1;
        xo_lo[g0 + (size_t)k * pitch] = l.b1;
      }
    }
    h.shift();
    l.shift();
  }
  return acc;
}

template <int SK>
__global__ void __launch_bounds__(NT) k_residual(const __grid_constant__ ResMaps M, const ProbDev* __restrict__ probs,
                                                 ProbState* __restrict__ state, float* __restrict__ partials,
                                                 int ntiles_max, float rtol, int max_cycles,
                                                 const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[0];
  const int n = L.n;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx;
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float XH[RES_H * XW];
  __shared__ __align__(128) float XL[RES_H * XW];
  __shared__ __align__(128) float BB[TB * TB];
  __shared__ __align__(8) uint64_t bar;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, (2 * RES_H * XW + TB * TB) * sizeof(float));
    tma_load_3d(XH, &M.xh, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(XL, &M.xl, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(BB, &M.b, &bar, C0, R0, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  const float acc = inner_tile(R0, C0, n) ? residual_tile<SK, true>(L, s, XH, XL, BB, R0, C0, L.r)
                                          : residual_tile<SK, false>(L, s, XH, XL, BB, R0, C0, L.r);
  float rhi, rlo;
  if (block_partial_and_last<NT>(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, rhi, rlo)) {
    if (threadIdx.x == 0) decide(state[p], rhi, rlo, rtol, max_cycles);
  }
}

// ---------------------------------------------------------------------- k_down
// e = H r (pre-smoothing from zero) on rows/cols R0-1 .. R0+33, s = r - A e on R0 .. R0+32
// (over r in place), r_c = P^T s on the tile's 16 x 16 coarse points.  Threads walk
// vertical strips of 5 rows with a 3x3 register window.
template <int SK, int HK, bool IN>
__device__ __forceinline__ void down_tile(const LevelDev& L, const float (&s)[9], const float* wtab,
                                          const float (&wi)[9], float omega, float* rs, float* es, float* eo,
                                          int R0, int C0) {
  constexpr int KS = 5;
  const int n = L.n, t = threadIdx.x;
  {
    constexpr int NS = (ES + KS - 1) / KS;
    if (t < ES * NS) {
      const int tj = t % ES, t0 = (t / ES) * KS, j = C0 - 1 + tj;
      const bool own_col = (unsigned)(tj - 1) < (unsigned)TB;
      const float* c = rs + (t0 + 1) * XW + tj + 3;
      Win v;
      if (HK != HK_JACOBI) v.load_ab(c, XW);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int ti = t0 + k;
        if (ES % KS == 0 || ti < ES) {
          const int i = R0 - 1 + ti;
          if (HK != HK_JACOBI) v.load_c(c + k * XW, XW);
          else v.b1 = c[k * XW];
          float e = 0.f;
          if (IN || inside(i, j, n)) e = tapply_H<SK, HK, IN>(L, s, wtab, wi, omega, i, j, v);
          es[ti * ESP + tj] = e;
          if (own_col && (unsigned)(ti - 1) < (unsigned)TB) eo[(ti - 1) * TB + tj - 1] = e;
          if (HK != HK_JACOBI) v.shift();
        }
      }
    }
  }
  fence_async_smem();
  __syncthreads();
  {
    constexpr int W2 = TB + 1, NS = (W2 + KS - 1) / KS;
    if (t < W2 * NS) {
      const int tj = t % W2, t0 = (t / W2) * KS, j = C0 + tj;
      const float* c = es + (t0 + 1) * ESP + tj + 1;
      float* rp = rs + (t0 + 2) * XW + tj + 4;
      Win v;
      v.load_ab(c, ESP);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int ti = t0 + k;
        if (ti < W2) {
          const int i = R0 + ti;
          v.load_c(c + k * ESP, ESP);
          float sv = 0.f;
          if (IN || inside(i, j, n)) sv = rp[k * XW] - tapply_A<SK>(L, s, i, j, v);
          rp[k * XW] = sv;
          v.shift();
        }
      }
    }
  }
  __syncthreads();
}

template <int SK, int HK>
__global__ void __launch_bounds__(NT, SK == SK_CONST ? 8 : 6) k_down(const __grid_constant__ DownMaps M, const ProbDev* __restrict__ probs,
                                             ProbState* __restrict__ state, int l, float omega,
                                             const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int ntx = (n + TB - 1) / TB;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float rs[DN_H * XW];  // r, then s = r - A e in place
  __shared__ __align__(128) float eo[TB * TB];    // e on the owned points (stored by TMA)
  __shared__ __align__(128) float rco[TC * TC];   // r_c (stored by TMA)
  __shared__ float es[ES * ESP];
  __shared__ float wtab[HK == HK_TABLE ? 9 * MG_PROXY * MG_PROXY : 1];
  __shared__ __align__(8) uint64_t bar;
  const bool in = inner_tile(R0, C0, n);
  float s[9], wi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  if (HK == HK_TABLE) load_table(L, in, wtab, wi);
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, DN_H * XW * sizeof(float));
    tma_load_3d(rs, &M.r, &bar, C0 - 4, R0 - 2, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  if (in) down_tile<SK, HK, true>(L, s, wtab, wi, omega, rs, es, eo, R0, C0);
  else down_tile<SK, HK, false>(L, s, wtab, wi, omega, rs, es, eo, R0, C0);
  if (threadIdx.x == 0) tma_store_3d(&M.e, eo, C0, R0, p);
  {
    const int a = threadIdx.x >> 4, b = threadIdx.x & 15;
    rco[a * TC + b] = restrict_at(rs + (2 * a + 3) * XW + 2 * b + 5, XW);
  }
  fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    tma_store_3d(&M.rc, rco, C0 / 2, R0 / 2, p);
    tma_store_commit();
    tma_store_wait();
  }
}

// ------------------------------------------------------------------------ k_up
// e1 = e + P e_c on rows/cols R0-2 .. R0+33 (zero outside the grid without masking: e and
// e_c are zero-filled there), t = r - A e1 on R0-1 .. R0+32, e = e1 + H t on the tile; on
// level 0 e is added to the float-float iterate.
template <int SK, int HK, bool UPDX, bool IN>
__device__ __forceinline__ void up_tile(const LevelDev& L, const float (&s)[9], const float* wtab,
                                        const float (&wi)[9], float omega, float* es, float* rs, const float* ecs,
                                        const float* xhs, const float* xls, float* xhi, float* xlo, int p, int R0,
                                        int C0) {
  const int n = L.n, pitch = L.pitch, t = threadIdx.x;
  {
    // bilinear P: P e_c(i, j) = ((c(ia,ja) + c(ia,jb)) + (c(ib,ja) + c(ib,jb))) / 4 with
    // ia = floor((i-1)/2), ib = floor(i/2) (equal for odd i), ja, jb likewise
    constexpr int W1 = TB + 4, KS = 6, NS = W1 / KS;
    if (t < W1 * NS) {
      const int tj = t % W1, t0 = (t / W1) * KS, j = C0 - 2 + tj;
      const int I0 = R0 / 2 - 2, J0 = C0 / 2 - 4;
      const int ja = ((j - 1) >> 1) - J0, jb = (j >> 1) - J0;
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int ti = t0 + k, i = R0 - 2 + ti;
        const float* ra = ecs + (((i - 1) >> 1) - I0) * EC_W;
        const float* rb = ecs + ((i >> 1) - I0) * EC_W;
        es[ti * XW + tj + 2] += 0.25f * ((ra[ja] + ra[jb]) + (rb[ja] + rb[jb]));
      }
    }
  }
  __syncthreads();
  {
    constexpr int W2 = TB + 2, KS = 5, NS = (W2 + KS - 1) / KS;
    if (t < W2 * NS) {
      const int tj = t % W2, t0 = (t / W2) * KS, j = C0 - 1 + tj;
      const float* c = es + (t0 + 1) * XW + tj + 3;
      float* rp = rs + t0 * XW + tj + 3;
      Win v;
      v.load_ab(c, XW);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int ti = t0 + k;
        if (ti < W2) {
          const int i = R0 - 1 + ti;
          v.load_c(c + k * XW, XW);
          float tv = 0.f;
          if (IN || inside(i, j, n)) tv = rp[k * XW] - tapply_A<SK>(L, s, i, j, v);
          rp[k * XW] = tv;
          v.shift();
        }
      }
    }
  }
  __syncthreads();
  {
    constexpr int KS = TB / NW;
    const int tj = threadIdx.x & 31, t0 = (threadIdx.x >> 5) * KS, j = C0 + tj;
    const float* c = rs + (t0 + 1) * XW + tj + 4;
    const float* e1 = es + (t0 + 2) * XW + tj + 4;
    Win v;
    if (HK != HK_JACOBI) v.load_ab(c, XW);
    const size_t row0 = (size_t)(R0 + t0) * pitch + j;
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int i = R0 + t0 + k;
      if (HK != HK_JACOBI) v.load_c(c + k * XW, XW);
      else v.b1 = c[k * XW];
      if (IN || inside(i, j, n)) {
        const float e = e1[k * XW] + tapply_H<SK, HK, IN>(L, s, wtab, wi, omega, i, j, v);
        if (UPDX) {
          const size_t g = (size_t)p * n * pitch + row0 + (size_t)k * pitch;
          float hi = xhs[(t0 + k) * TB + tj], lo = xls[(t0 + k) * TB + tj], sum, err;
          two_sum(hi, e, sum, err);
          err += lo;
          fast_two_sum(sum, err, hi, lo);
          xhi[g] = hi;
          xlo[g] = lo;
        } else {
          L.f[row0 + (size_t)k * pitch] = e;  // e is still read with halos by other CTAs
        }
      }
      if (HK != HK_JACOBI) v.shift();
    }
  }
}

template <int SK, int HK, bool UPDX>
__global__ void __launch_bounds__(NT, SK == SK_CONST ? 8 : 6) k_up(const __grid_constant__ UpMaps M, const ProbDev* __restrict__ probs,
                                           ProbState* __restrict__ state, int l, float omega, float* __restrict__ xhi,
                                           float* __restrict__ xlo, const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int ntx = (n + TB - 1) / TB;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float es[UPE_H * XW];   // e, then e1 = e + P e_c in place
  __shared__ __align__(128) float rs[UPR_H * XW];   // r, then t = r - A e1 in place
  __shared__ __align__(128) float ecs[EC_H * EC_W];
  __shared__ __align__(128) float xhs[UPDX ? TB * TB : 4];
  __shared__ __align__(128) float xls[UPDX ? TB * TB : 4];
  __shared__ float wtab[HK == HK_TABLE ? 9 * MG_PROXY * MG_PROXY : 1];
  __shared__ __align__(8) uint64_t bar;
  const bool in = inner_tile(R0, C0, n);
  float s[9], wi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  if (HK == HK_TABLE) load_table(L, in, wtab, wi);
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, ((UPE_H + UPR_H) * XW + EC_H * EC_W + (UPDX ? 2 * TB * TB : 0)) * sizeof(float));
    tma_load_3d(es, &M.e, &bar, C0 - 4, R0 - 2, p);
    tma_load_3d(rs, &M.r, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(ecs, &M.ec, &bar, C0 / 2 - 4, R0 / 2 - 2, p);
    if (UPDX) {
      tma_load_3d(xhs, &M.xh, &bar, C0, R0, p);
      tma_load_3d(xls, &M.xl, &bar, C0, R0, p);
    }
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  if (in) up_tile<SK, HK, UPDX, true>(L, s, wtab, wi, omega, es, rs, ecs, xhs, xls, xhi, xlo, p, R0, C0);
  else up_tile<SK, HK, UPDX, false>(L, s, wtab, wi, omega, es, rs, ecs, xhs, xls, xhi, xlo, p, R0, C0);
}

// ----------------------------------------------------------------- k_up0
// Level 0: the up-sweep of k_up computed one point wider (e1 on rows/cols R0-3 .. R0+34,
// t on R0-2 .. R0+33, e on R0-1 .. R0+32), the float-float update of x on the tile and its
// halo in shared memory, then the compensated residual of the new iterate on the tile,
// the norm partial and the stopping test: the residual of the next cycle without
// re-reading x.
template <int SK, int HK, bool IN>
__device__ __forceinline__ void up0_tile(const LevelDev& L, const float (&s)[9], const float* wtab,
                                         const float (&wi)[9], float omega, float* es, float* rs, const float* ecs,
                                         float* xh, float* xl, int R0, int C0) {
  const int n = L.n, t = threadIdx.x;
  {
    // e1 = e + P e_c in strips of 8 fine rows starting on even offsets: strip s8 reads
    // coarse rows 4 s8 .. 4 s8 + 4, so every row index below is a compile-time constant
    constexpr int W1 = TB + 6, KS = 8, NS = (W1 + KS - 1) / KS;
    if (t < W1 * NS) {
      const int tj = t % W1, s8 = t / W1, j = C0 - 3 + tj;
      const int J0 = C0 / 2 - 4;
      const int ja = ((j - 1) >> 1) - J0, jb = (j >> 1) - J0;
      const float* cb = ecs + 4 * s8 * EC_W;
      float* ep = es + 8 * s8 * XW + tj + 1;
      if (s8 < NS - 1) {
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          const float* ra = cb + (k >> 1) * EC_W;
          const float* rb = cb + ((k + 1) >> 1) * EC_W;
          ep[k * XW] += 0.25f * ((ra[ja] + ra[jb]) + (rb[ja] + rb[jb]));
        }
      } else {
#pragma unroll
        for (int k = 0; k < W1 - KS * (NS - 1); ++k) {
          const float* ra = cb + (k >> 1) * EC_W;
          const float* rb = cb + ((k + 1) >> 1) * EC_W;
          ep[k * XW] += 0.25f * ((ra[ja] + ra[jb]) + (rb[ja] + rb[jb]));
        }
      }
    }
  }
  __syncthreads();
  {
    constexpr int W2 = TB + 4, KS = 6, NS = W2 / KS;
    if (t < W2 * NS) {
      const int tj = t % W2, t0 = (t / W2) * KS, j = C0 - 2 + tj;
      const float* c = es + (t0 + 1) * XW + tj + 2;
      float* rp = rs + t0 * XW + tj + 2;
      Win v;
      v.load_ab(c, XW);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int i = R0 - 2 + t0 + k;
        v.load_c(c + k * XW, XW);
        float tv = 0.f;
        if (IN || inside(i, j, n)) tv = rp[k * XW] - tapply_A<SK>(L, s, i, j, v);
        rp[k * XW] = tv;
        v.shift();
      }
    }
  }
  __syncthreads();
  {
    constexpr int W3 = TB + 2, KS = 5, NS = (W3 + KS - 1) / KS;
    if (t < W3 * NS) {
      const int tj = t % W3, t0 = (t / W3) * KS, j = C0 - 1 + tj;
      const float* c = rs + (t0 + 1) * XW + tj + 3;
      const float* e1 = es + (t0 + 2) * XW + tj + 3;
      float* ph = xh + t0 * XW + tj + 3;
      float* pl = xl + t0 * XW + tj + 3;
      Win v;
      if (HK != HK_JACOBI) v.load_ab(c, XW);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int ti = t0 + k, i = R0 - 1 + ti;
        if (ti < W3) {
          if (HK != HK_JACOBI) v.load_c(c + k * XW, XW);
          else v.b1 = c[k * XW];
          if (IN || inside(i, j, n)) {
            const float e = e1[k * XW] + tapply_H<SK, HK, IN>(L, s, wtab, wi, omega, i, j, v);
            float hi = ph[k * XW], lo = pl[k * XW], sum, err;
            two_sum(hi, e, sum, err);
            err += lo;
            fast_two_sum(sum, err, hi, lo);
            ph[k * XW] = hi;
            pl[k * XW] = lo;
          }
          if (HK != HK_JACOBI) v.shift();
        }
      }
    }
  }
  __syncthreads();
}

template <int SK, int HK>
__global__ void __launch_bounds__(NT, SK == SK_CONST ? 8 : 4) k_up0(const __grid_constant__ Up0Maps M, const ProbDev* __restrict__ probs,
                                            ProbState* __restrict__ state, float* __restrict__ partials,
                                            int ntiles_max, float omega, float rtol, int max_cycles,
                                            float* __restrict__ xhi, float* __restrict__ xlo,
                                            float* __restrict__ rnew, const float* __restrict__ b0,
                                            const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[0];
  const int n = L.n;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx;
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float es[UP0E_H * XW];  // e, then e1 = e + P e_c in place
  __shared__ __align__(128) float rs[UP0R_H * XW];  // r, then t = r - A e1 in place
  __shared__ __align__(128) float ecs[EC0_H * EC_W];
  __shared__ __align__(128) float xh[RES_H * XW];   // x on the tile and its halo, updated in place
  __shared__ __align__(128) float xl[RES_H * XW];
  __shared__ __align__(8) uint64_t bar;
  const bool in = inner_tile(R0, C0, n);
  float s[9], wi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  // Edge tiles read the class table through L1 and the residual reads b from global memory
  // (no shared copies: 28.7 KB per CTA, 8 CTAs fit on an SM)
  const float* wtab = L.W;
  if (HK == HK_TABLE && in) {
#pragma unroll
    for (int k = 0; k < 9; ++k) wi[k] = L.W[k * L.T * L.T + MG_NET_MARGIN * L.T + MG_NET_MARGIN];
  }
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, ((UP0E_H + UP0R_H + 2 * RES_H) * XW + EC0_H * EC_W) * sizeof(float));
    tma_load_3d(es, &M.e, &bar, C0 - 4, R0 - 3, p);
    tma_load_3d(rs, &M.r, &bar, C0 - 4, R0 - 2, p);
    tma_load_3d(ecs, &M.ec, &bar, C0 / 2 - 4, R0 / 2 - 2, p);
    tma_load_3d(xh, &M.x.xh, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(xl, &M.x.xl, &bar, C0 - 4, R0 - 1, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  if (in) up0_tile<SK, HK, true>(L, s, wtab, wi, omega, es, rs, ecs, xh, xl, R0, C0);
  else up0_tile<SK, HK, false>(L, s, wtab, wi, omega, es, rs, ecs, xh, xl, R0, C0);
  const size_t po = (size_t)p * n * L.pitch;
  const float acc = in ? residual_tile<SK, true>(L, s, xh, xl, nullptr, R0, C0, rnew + po, xhi + po, xlo + po, b0 + po)
                       : residual_tile<SK, false>(L, s, xh, xl, nullptr, R0, C0, rnew + po, xhi + po, xlo + po, b0 + po);
  float rhi, rlo;
  if (block_partial_and_last<NT>(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, rhi, rlo)) {
    if (threadIdx.x == 0) decide(state[p], rhi, rlo, rtol, max_cycles);
  }
}

// ------------------------------------------------------------ k_up0 in pairs
// The constant-stencil level-0 kernel with two adjacent columns per thread (128 threads per
// 32 x 32 tile, the same copies and phases as k_up0).  A pair's two values share one
// 64-bit register pair and every arithmetic step is one packed FP32 instruction (add, mul,
// fma on .f32x2; each lane rounded exactly as the scalar instruction), and the four columns
// c-1 .. c+2 of a window row around the pair (c, c+1) are two aligned 64-bit shared loads
// when c is odd.  Half the threads with twice the registers each keep 8 CTAs per SM.
constexpr int NTP = 128;

// H v for the pair at (i, j), (i, j+1): Jacobi, or the interior kernel on inner tiles, else
// each point's class kernel (points outside the grid have no class: 0 there)
template <int HK, bool IN, bool ODD>
__device__ __forceinline__ float2 tapply_H2(const LevelDev& L, const float (&s)[9], const float* wtab,
                                            const float (&wi)[9], float omega, int i, int j, const Win2& v) {
  if (HK == HK_JACOBI) return mul2(p2(omega / s[4]), v.mb);
  if (IN) return dot9w<ODD>(wi, v);
  float2 h = p2(0.f);
  if (inside(i, j, L.n)) h.x = tapply_H<SK_CONST, HK, false>(L, s, wtab, wi, omega, i, j, lane_win(v, 0));
  if (inside(i, j + 1, L.n)) h.y = tapply_H<SK_CONST, HK, false>(L, s, wtab, wi, omega, i, j + 1, lane_win(v, 1));
  return h;
}

// zero the lanes of a pair that lie outside the grid (edge tiles)
__device__ __forceinline__ float2 mask2(float2 v, int i, int j, int n) {
  if (!inside(i, j, n)) v.x = 0.f;
  if (!inside(i, j + 1, n)) v.y = 0.f;
  return v;
}

template <int HK, bool IN>
__device__ __forceinline__ void up0p_tile(const LevelDev& L, const float (&s)[9], const float* wtab,
                                          const float (&wi)[9], float omega, float* es, float* rs, const float* ecs,
                                          float* xh, float* xl, int R0, int C0) {
  const int n = L.n, t = threadIdx.x;
  {
    // e1 = e + P e_c on rows R0-3 .. R0+34 and the whole box width: pair q is box columns
    // 2q, 2q+1 (grid columns C0-4+2q, even, and the odd one after it), whose bilinear
    // weights read coarse box columns (q+1, q+2) and (q+2, q+2).  Strips of 8 fine rows
    // from even offsets read coarse rows 4 s .. 4 s + 4 (a coarse row pair sum serves two
    // fine rows).
    constexpr int NQ = XW / 2, KS = 8, NS = (UP0E_H + KS - 1) / KS, LAST = UP0E_H - KS * (NS - 1);
    if (t < NQ * NS) {
      const int q = t % NQ, s8 = t / NQ;
      const float* cb = ecs + 4 * s8 * EC_W + q + 1;
      float* ep = es + 8 * s8 * XW + 2 * q;
      float2 S[KS / 2 + 1];
      if (s8 < NS - 1) {
#pragma unroll
        for (int m = 0; m <= KS / 2; ++m) {
          const float a = cb[m * EC_W], b = cb[m * EC_W + 1];
          S[m] = add2(make_float2(a, b), p2(b));
        }
#pragma unroll
        for (int k = 0; k < KS; ++k) st2(ep + k * XW, fma2(p2(0.25f), add2(S[k >> 1], S[(k + 1) >> 1]), ld2(ep + k * XW)));
      } else {
#pragma unroll
        for (int m = 0; m <= LAST / 2; ++m) {
          const float a = cb[m * EC_W], b = cb[m * EC_W + 1];
          S[m] = add2(make_float2(a, b), p2(b));
        }
#pragma unroll
        for (int k = 0; k < LAST; ++k) st2(ep + k * XW, fma2(p2(0.25f), add2(S[k >> 1], S[(k + 1) >> 1]), ld2(ep + k * XW)));
      }
    }
  }
  __syncthreads();
  {
    // t = r - A e1 on rows R0-2 .. R0+33, box columns 1 .. 38 (pair q: 2q+1, 2q+2), 9-row strips
    constexpr int NQ = (XW - 2) / 2, KS = 9, NS = UP0R_H / KS;
    static_assert(KS * NS == UP0R_H && 16 * NS + (NQ - 16) * NS <= NTP, "phase t");
    int q, sb;
    if (chunk_item<NQ, NS>(t, q, sb)) {
      const int t0 = sb * KS, j = C0 - 3 + 2 * q;
      const float* c = es + t0 * XW + 2 * q;  // column 2q = c-1 of row t0 (window row a)
      float* rp = rs + t0 * XW + 2 * q + 1;
      Win2 v;
      row_odd(c, v.la, v.ma, v.ra);
      row_odd(c + XW, v.lb, v.mb, v.rb);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        row_odd(c + (k + 2) * XW, v.lc, v.mc, v.rc);
        float2 tv = sub2(make_float2(rp[k * XW], rp[k * XW + 1]), dot9w<true>(s, v));
        if (!IN) tv = mask2(tv, R0 - 2 + t0 + k, j, n);
        rp[k * XW] = tv.x;
        rp[k * XW + 1] = tv.y;
        v.shift();
      }
    }
  }
  __syncthreads();
  {
    // e = e1 + H t and the float-float update of x on rows R0-1 .. R0+32, box columns
    // 2 .. 37 (pair q: 2q+2, 2q+3; the residual reads 3 .. 36), 5-row strips; outside the
    // grid x keeps its zero
    constexpr int NQ = (TB + 4) / 2, KS = 5, NS = (RES_H + KS - 1) / KS;
    static_assert(16 * NS + (NQ - 16) * NS <= NTP, "phase e");
    int q, sc;
    if (chunk_item<NQ, NS>(t, q, sc)) {
      const int t0 = sc * KS, j = C0 - 2 + 2 * q;
      const float* c = rs + t0 * XW + 2 * q + 2;  // column c of window row a
      const float* e1 = es + (t0 + 2) * XW + 2 * q + 2;
      float* ph = xh + t0 * XW + 2 * q + 2;
      float* pl = xl + t0 * XW + 2 * q + 2;
      Win2 v;
      if (HK != HK_JACOBI) {
        row_even(c, v.la, v.ma, v.ra);
        row_even(c + XW, v.lb, v.mb, v.rb);
      }
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int ti = t0 + k, i = R0 - 1 + ti;
        if (ti < RES_H) {
          if (HK != HK_JACOBI) row_even(c + (k + 2) * XW, v.lc, v.mc, v.rc);
          else v.mb = ld2(c + (k + 1) * XW);
          const float2 e = add2(ld2(e1 + k * XW), tapply_H2<HK, IN, false>(L, s, wtab, wi, omega, i, j, v));
          float2 sum, err, hi, lo;
          two_sum2(ld2(ph + k * XW), e, sum, err);
          err = add2(err, ld2(pl + k * XW));
          fast_two_sum2(sum, err, hi, lo);
          if (IN) {
            st2(ph + k * XW, hi);
            st2(pl + k * XW, lo);
          } else {
            if (inside(i, j, n)) {
              ph[k * XW] = hi.x;
              pl[k * XW] = lo.x;
            }
            if (inside(i, j + 1, n)) {
              ph[k * XW + 1] = hi.y;
              pl[k * XW + 1] = lo.y;
            }
          }
          if (HK != HK_JACOBI) v.shift();
        }
      }
    }
  }
  __syncthreads();
}

// The compensated residual r = b - A (x_hi + x_lo) of the new iterate on the tile (pair q:
// grid columns C0+2q, C0+2q+1; 4-row strips), stored with the iterate; returns this
// thread's share of ||r||^2.
template <bool IN>
__device__ __forceinline__ float residual_pair(const LevelDev& L, const float (&s)[9], const float* XH,
                                               const float* XL, int R0, int C0, float* rdst, float* xo_hi,
                                               float* xo_lo, const float* bg) {
  constexpr int NQ = TB / 2, KS = TB / (NTP / NQ);
  const int n = L.n, pitch = L.pitch;
  const int q = threadIdx.x % NQ, t0 = (threadIdx.x / NQ) * KS, j = C0 + 2 * q;
  const float* ch = XH + t0 * XW + 2 * q + 4;  // column c of window row a
  const float* cl = XL + t0 * XW + 2 * q + 4;
  Win2 h, l;
  row_even(ch, h.la, h.ma, h.ra);
  row_even(cl, l.la, l.ma, l.ra);
  row_even(ch + XW, h.lb, h.mb, h.rb);
  row_even(cl + XW, l.lb, l.mb, l.rb);
  float2 acc = p2(0.f);
  const size_t g0 = (size_t)(R0 + t0) * pitch + j;
  // b of all the thread's rows first, so that their latencies overlap
  float2 bv[KS];
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const int i = R0 + t0 + k;
    const size_t g = g0 + (size_t)k * pitch;
    if (IN) bv[k] = __ldg(reinterpret_cast<const float2*>(bg + g));
    else bv[k] = make_float2(inside(i, j, n) ? __ldg(bg + g) : 0.f, inside(i, j + 1, n) ? __ldg(bg + g + 1) : 0.f);
  }
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    row_even(ch + (k + 2) * XW, h.lc, h.mc, h.rc);
    row_even(cl + (k + 2) * XW, l.lc, l.mc, l.rc);
    const int i = R0 + t0 + k;
    const size_t g = g0 + (size_t)k * pitch;
    const bool in0 = IN || inside(i, j, n), in1 = IN || inside(i, j + 1, n);
    float2 hi = bv[k];
    float2 lo = p2(0.f);
    dot2_sub2(s[0], h.la, l.la, hi, lo);
    dot2_sub2(s[1], h.ma, l.ma, hi, lo);
    dot2_sub2(s[2], h.ra, l.ra, hi, lo);
    dot2_sub2(s[3], h.lb, l.lb, hi, lo);
    dot2_sub2(s[4], h.mb, l.mb, hi, lo);
    dot2_sub2(s[5], h.rb, l.rb, hi, lo);
    dot2_sub2(s[6], h.lc, l.lc, hi, lo);
    dot2_sub2(s[7], h.mc, l.mc, hi, lo);
    dot2_sub2(s[8], h.rc, l.rc, hi, lo);
    float2 r = add2(hi, lo);
    if (IN) {
      st2(rdst + g, r);
      st2(xo_hi + g, h.mb);
      st2(xo_lo + g, l.mb);
    } else {
      if (in0) {
        rdst[g] = r.x;
        xo_hi[g] = h.mb.x;
        xo_lo[g] = l.mb.x;
      } else {
        r.x = 0.f;
      }
      if (in1) {
        rdst[g + 1] = r.y;
        xo_hi[g + 1] = h.mb.y;
        xo_lo[g + 1] = l.mb.y;
      } else {
        r.y = 0.f;
      }
    }
    acc = fma2(r, r, acc);
    h.shift();
    l.shift();
  }
  return acc.x + acc.y;
}

template <int HK>
__global__ void __launch_bounds__(NTP, 8) k_up0p(const __grid_constant__ Up0Maps M, const ProbDev* __restrict__ probs,
                                                 ProbState* __restrict__ state, float* __restrict__ partials,
                                                 int ntiles_max, float omega, float rtol, int max_cycles,
                                                 float* __restrict__ xhi, float* __restrict__ xlo,
                                                 float* __restrict__ rnew, const float* __restrict__ b0,
                                                 const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[0];
  const int n = L.n;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx;
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float es[UP0E_H * XW];
  __shared__ __align__(128) float rs[UP0R_H * XW];
  __shared__ __align__(128) float ecs[EC0_H * EC_W];
  __shared__ __align__(128) float xh[RES_H * XW];
  __shared__ __align__(128) float xl[RES_H * XW];
  __shared__ __align__(8) uint64_t bar;
  const bool in = inner_tile(R0, C0, n);
  float s[9], wi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = L.s[k];
  const float* wtab = L.W;
  if (HK == HK_TABLE && in) {
#pragma unroll
    for (int k = 0; k < 9; ++k) wi[k] = L.W[k * L.T * L.T + MG_NET_MARGIN * L.T + MG_NET_MARGIN];
  }
  // b is read from global memory in the residual at the end: bring its tile to L2 now
  if (threadIdx.x == 0) tma_prefetch_3d(&M.x.b, C0, R0, p);
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, ((UP0E_H + UP0R_H + 2 * RES_H) * XW + EC0_H * EC_W) * sizeof(float));
    tma_load_3d(es, &M.e, &bar, C0 - 4, R0 - 3, p);
    tma_load_3d(rs, &M.r, &bar, C0 - 4, R0 - 2, p);
    tma_load_3d(ecs, &M.ec, &bar, C0 / 2 - 4, R0 / 2 - 2, p);
    tma_load_3d(xh, &M.x.xh, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(xl, &M.x.xl, &bar, C0 - 4, R0 - 1, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  if (in) up0p_tile<HK, true>(L, s, wtab, wi, omega, es, rs, ecs, xh, xl, R0, C0);
  else up0p_tile<HK, false>(L, s, wtab, wi, omega, es, rs, ecs, xh, xl, R0, C0);
  const size_t po = (size_t)p * n * L.pitch;
  const float acc = in ? residual_pair<true>(L, s, xh, xl, R0, C0, rnew + po, xhi + po, xlo + po, b0 + po)
                       : residual_pair<false>(L, s, xh, xl, R0, C0, rnew + po, xhi + po, xlo + po, b0 + po);
  float rhi, rlo;
  if (block_partial_and_last<NTP>(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, rhi, rlo)) {
    if (threadIdx.x == 0) decide(state[p], rhi, rlo, rtol, max_cycles);
  }
}

// ------------------------------------------------------------ k_down in pairs
// k_down on constant stencils with two columns per thread (128 threads per tile) in packed
// FP32, like k_up0p.  e = H r goes to its own buffer with a column origin at box column 3,
// so that the odd box columns of the pre-smoothing pairs and the window rows of the
// residual pass are all aligned 64-bit shared accesses.
constexpr int EPW = 36;  // e buffer: box columns 3 .. 38, rows R0-1 .. R0+33

template <int HK, bool IN>
__device__ __forceinline__ void downp_tile(const LevelDev& L, const float (&s)[9], const float* wtab,
                                           const float (&wi)[9], float omega, float* rs, float* es, float* eo,
                                           int R0, int C0) {
  const int n = L.n, t = threadIdx.x;
  {
    // e = H r on rows R0-1 .. R0+33, box columns 3 .. 38 (pair q: 2q+3, 2q+4; the residual
    // reads 3 .. 37)
    constexpr int NQ = 18, KS = 5, NS = (ES + KS - 1) / KS;
    static_assert(16 * NS + (NQ - 16) * NS <= NTP, "phase e");
    int q, sa;
    if (chunk_item<NQ, NS>(t, q, sa)) {
      const int t0 = sa * KS, j = C0 - 1 + 2 * q;
      const float* c = rs + t0 * XW + 2 * q + 2;  // column c-1 of window row a
      Win2 v;
      if (HK != HK_JACOBI) {
        row_odd(c, v.la, v.ma, v.ra);
        row_odd(c + XW, v.lb, v.mb, v.rb);
      }
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int ti = t0 + k, i = R0 - 1 + ti;
        if (ES % KS == 0 || ti < ES) {
          if (HK != HK_JACOBI) row_odd(c + (k + 2) * XW, v.lc, v.mc, v.rc);
          else v.mb = make_float2(c[(k + 1) * XW + 1], c[(k + 1) * XW + 2]);
          float2 e = tapply_H2<HK, IN, true>(L, s, wtab, wi, omega, i, j, v);
          if (!IN) e = mask2(e, i, j, n);
          st2(es + ti * EPW + 2 * q, e);
          if (HK != HK_JACOBI) v.shift();
        }
      }
    }
  }
  __syncthreads();
  {
    // s = r - A e on rows R0 .. R0+32, box columns 4 .. 37 (pair q: 2q+4, 2q+5; the
    // restriction reads 4 .. 36), over r in place; the centre pair of each window row on
    // the tile is e at the pair's own points, which goes to eo (an aligned 64-bit store)
    // for the store of e
    constexpr int NQ = 17, KS = 5, NR = TB + 1, NS = (NR + KS - 1) / KS;
    static_assert(16 * NS + (NQ - 16) * NS <= NTP, "phase s");
    int q, sb;
    if (chunk_item<NQ, NS>(t, q, sb)) {
      const int t0 = sb * KS, j = C0 + 2 * q;
      const float* c = es + t0 * EPW + 2 * q;  // e box column 2q+3 = c-1 of window row a
      float* rp = rs + (t0 + 2) * XW + 2 * q + 4;
      Win2 v;
      row_odd(c, v.la, v.ma, v.ra);
      row_odd(c + EPW, v.lb, v.mb, v.rb);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int ti = t0 + k;
        if (ti < NR) {
          row_odd(c + (k + 2) * EPW, v.lc, v.mc, v.rc);
          float2 sv = sub2(ld2(rp + k * XW), dot9w<true>(s, v));
          if (!IN) sv = mask2(sv, R0 + ti, j, n);
          st2(rp + k * XW, sv);
          if (ti < TB && q < TB / 2) st2(eo + ti * TB + 2 * q, make_float2(v.lb.y, v.rb.x));
          v.shift();
        }
      }
    }
  }
  fence_async_smem();
  __syncthreads();
}

// A CTA takes `tpc` consecutive tiles of one problem through two r buffers: the copy of
// tile u+1 is in flight while tile u is computed, and the copy of tile u+2 starts as soon as
// tile u's buffer is free.
template <int HK>
__global__ void __launch_bounds__(NTP, 8) k_downp(const __grid_constant__ DownMaps M, const ProbDev* __restrict__ probs,
                                                  ProbState* __restrict__ state, int l, float omega, int tpc,
                                                  const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx;
  const int first = blockIdx.x * tpc;
  if (first >= ntiles) return;
  const int count = min(tpc, ntiles - first);
  // r, then s = r - A e in place; each buffer a whole number of 128-byte lines (the copy
  // engine writes to 128-byte aligned shared memory)
  constexpr int RSZ = (DN_H * XW + 31) / 32 * 32;
  __shared__ __align__(128) float rs[2][RSZ];
  __shared__ __align__(128) float eo[TB * TB];       // e on the owned points (stored by TMA)
  __shared__ __align__(128) float rco[TC * TC];      // r_c (stored by TMA)
  __shared__ __align__(16) float es[ES * EPW];
  __shared__ float wtab[HK == HK_TABLE ? 9 * MG_PROXY * MG_PROXY : 1];
  __shared__ __align__(8) uint64_t bar[2];
  float s[9], wi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = L.s[k];
  if (HK == HK_TABLE) {
    const int T = L.T, Mg = MG_NET_MARGIN;
#pragma unroll
    for (int k = 0; k < 9; ++k) wi[k] = L.W[k * T * T + Mg * T + Mg];
    bool edge = false;
    for (int u = 0; u < count; ++u) edge |= !inner_tile(((first + u) / ntx) * TB, ((first + u) % ntx) * TB, n);
    if (edge)
      for (int k = threadIdx.x; k < 9 * T * T; k += NTP) wtab[k] = L.W[k];
  }
  pdl_wait();
  if (!st_active(state + p)) return;
  // thread 0: the copy of tile u into buffer u & 1
  auto issue = [&](int u) {
    const int tt = first + u;
    mbar_arrive_expect_tx(&bar[u & 1], DN_H * XW * sizeof(float));
    tma_load_3d(rs[u & 1], &M.r, &bar[u & 1], (tt % ntx) * TB - 4, (tt / ntx) * TB - 2, p);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    issue(0);
    if (count > 1) issue(1);
  }
  __syncthreads();
  for (int u = 0; u < count; ++u) {
    const int tt = first + u, R0 = (tt / ntx) * TB, C0 = (tt % ntx) * TB;
    const bool in = inner_tile(R0, C0, n);
    float* r = rs[u & 1];
    // the stores of the previous tile have read eo and rco before they are written again
    if (u > 0 && threadIdx.x == 0) tma_store_wait_read();
    const bool more = u + 1 < count;
    if (!tile_wait_phase(&bar[u & 1], (u >> 1) & 1, more ? &bar[(u + 1) & 1] : nullptr, ((u + 1) >> 1) & 1, state[p])) {
      if (threadIdx.x == 0) tma_store_wait();
      return;
    }
    if (in) downp_tile<HK, true>(L, s, wtab, wi, omega, r, es, eo, R0, C0);
    else downp_tile<HK, false>(L, s, wtab, wi, omega, r, es, eo, R0, C0);
    if (threadIdx.x == 0) tma_store_3d(&M.e, eo, C0, R0, p);
    {
      // r_c = P^T s: coarse column b = lane of a half-warp, coarse rows a and a + 8 (fine
      // rows 2a .. 2a+2 and columns 2b .. 2b+2 of the tile: one 64-bit and one single load
      // per row), the order of restrict_at
      const int bq = threadIdx.x & 15, a0 = threadIdx.x >> 4;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int a = a0 + 8 * h;
        const float* c = r + (2 * a + 2) * XW + 2 * bq + 4;
        float2 u[3];
        float z[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          u[q] = ld2(c + q * XW);
          z[q] = c[q * XW + 2];
        }
        const float edge = (u[0].y + u[2].y) + (u[1].x + z[1]);
        const float corner = (u[0].x + z[0]) + (u[2].x + z[2]);
        rco[a * TC + bq] = u[1].y + 0.5f * edge + 0.25f * corner;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tma_store_3d(&M.rc, rco, C0 / 2, R0 / 2, p);
      tma_store_commit();
      if (u + 2 < count) issue(u + 2);  // every thread is done with buffer u & 1
    }
  }
  if (threadIdx.x == 0) tma_store_wait();
}

// ------------------------------------------------------- k_update_residual
// The level-0 end of a cycle whose up-sweep ran in other kernels (the linear smoother's
// path): x += e_0 in float-float on the tile and its one-point halo in shared memory, then
// the compensated residual of the new iterate on the tile (storing the new iterate), its
// norm partial and, in the last CTA of a problem, the stopping test.
template <int SK>
__global__ void __launch_bounds__(NT) k_update_residual(const __grid_constant__ ResMaps X,
                                                        const __grid_constant__ CUtensorMap E,
                                                        const ProbDev* __restrict__ probs, ProbState* __restrict__ state,
                                                        float* __restrict__ partials, int ntiles_max, float rtol,
                                                        int max_cycles, float* __restrict__ xhi, float* __restrict__ xlo,
                                                        float* __restrict__ rnew, const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[0];
  const int n = L.n;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx;
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float xh[RES_H * XW];
  __shared__ __align__(128) float xl[RES_H * XW];
  __shared__ __align__(128) float es[RES_H * XW];
  __shared__ __align__(128) float bb[TB * TB];
  __shared__ __align__(8) uint64_t bar;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, (3 * RES_H * XW + TB * TB) * sizeof(float));
    tma_load_3d(xh, &X.xh, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(xl, &X.xl, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(es, &E, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(bb, &X.b, &bar, C0, R0, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  // the box is zero outside the grid in all three arrays, so the update keeps it zero there
  for (int q = threadIdx.x; q < RES_H * XW; q += NT) {
    float hi = xh[q], lo = xl[q], sum, err;
    two_sum(hi, es[q], sum, err);
    err += lo;
    fast_two_sum(sum, err, hi, lo);
    xh[q] = hi;
    xl[q] = lo;
  }
  __syncthreads();
  const size_t po = (size_t)p * n * L.pitch;
  const float acc = inner_tile(R0, C0, n)
                        ? residual_tile<SK, true>(L, s, xh, xl, bb, R0, C0, rnew + po, xhi + po, xlo + po)
                        : residual_tile<SK, false>(L, s, xh, xl, bb, R0, C0, rnew + po, xhi + po, xlo + po);
  float rhi, rlo;
  if (block_partial_and_last<NT>(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, rhi, rlo)) {
    if (threadIdx.x == 0) decide(state[p], rhi, rlo, rtol, max_cycles);
  }
}

// ------------------------------------------------------------ k_up in pairs
// k_up on constant stencils (levels >= 1) with two columns per thread (128 threads): e1 =
// e + P e_c over the whole box width in 8-row strips of pairs (a coarse row's pair sum serves
// two fine rows), t = r - A e1 on even pairs (the pair's r and t are 64-bit accesses), then
// e1 + H t on the tile's pairs, written to the level's array of its own (f).
template <int HK, bool IN>
__device__ __forceinline__ void upp_tile(const LevelDev& L, const float (&s)[9], const float* wtab,
                                         const float (&wi)[9], float omega, float* es, float* rs, const float* ecs,
                                         int R0, int C0) {
  const int n = L.n, t = threadIdx.x;
  {
    // e1 on rows R0-2 .. R0+33 (es row rr: fine row 2m reads coarse box rows m, m+1, row
    // 2m+1 coarse row m+1 twice) and box columns 0 .. 39 (pair q: coarse box columns
    // (q+1, q+2) and (q+2, q+2), as in k_up0p)
    constexpr int NQ = XW / 2, KS = 8, NS = (UPE_H + KS - 1) / KS, LAST = UPE_H - KS * (NS - 1);
    if (t < NQ * NS) {
      const int q = t % NQ, s8 = t / NQ;
      const float* cb = ecs + 4 * s8 * EC_W + q + 1;
      float* ep = es + KS * s8 * XW + 2 * q;
      float2 S[KS / 2 + 1];
      if (s8 < NS - 1) {
#pragma unroll
        for (int m = 0; m <= KS / 2; ++m) {
          const float a = cb[m * EC_W], b = cb[m * EC_W + 1];
          S[m] = add2(make_float2(a, b), p2(b));
        }
#pragma unroll
        for (int k = 0; k < KS; ++k)
          st2(ep + k * XW, fma2(p2(0.25f), add2(S[(k + 1) >> 1], S[(k >> 1) + 1]), ld2(ep + k * XW)));
      } else {
#pragma unroll
        for (int m = 0; m <= LAST / 2; ++m) {
          const float a = cb[m * EC_W], b = cb[m * EC_W + 1];
          S[m] = add2(make_float2(a, b), p2(b));
        }
#pragma unroll
        for (int k = 0; k < LAST; ++k)
          st2(ep + k * XW, fma2(p2(0.25f), add2(S[(k + 1) >> 1], S[(k >> 1) + 1]), ld2(ep + k * XW)));
      }
    }
  }
  __syncthreads();
  {
    // t = r - A e1 on rows R0-1 .. R0+32, box columns 2 .. 37 (pair q: 2q+2, 2q+3)
    constexpr int NQ = (TB + 4) / 2, KS = 5, NS = (UPR_H + KS - 1) / KS;
    static_assert(16 * NS + (NQ - 16) * NS <= NTP, "phase t");
    int q, sb;
    if (chunk_item<NQ, NS>(t, q, sb)) {
      const int t0 = sb * KS, j = C0 - 2 + 2 * q;
      const float* c = es + t0 * XW + 2 * q + 2;  // column c of window row a
      float* rp = rs + t0 * XW + 2 * q + 2;
      Win2 v;
      row_even(c, v.la, v.ma, v.ra);
      row_even(c + XW, v.lb, v.mb, v.rb);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        if (UPR_H % KS == 0 || t0 + k < UPR_H) {
          row_even(c + (k + 2) * XW, v.lc, v.mc, v.rc);
          float2 tv = sub2(ld2(rp + k * XW), dot9w<false>(s, v));
          if (!IN) tv = mask2(tv, R0 - 1 + t0 + k, j, n);
          st2(rp + k * XW, tv);
          v.shift();
        }
      }
    }
  }
  __syncthreads();
  {
    // e1 + H t on the tile: pair q = grid columns C0 + 2q, C0 + 2q + 1, 4-row strips
    constexpr int KS = 4;
    const int q = t & 15, t0 = (t >> 4) * KS, j = C0 + 2 * q;
    const float* c = rs + t0 * XW + 2 * q + 4;
    const float* e1 = es + (t0 + 2) * XW + 2 * q + 4;
    float* out = L.f + (size_t)(R0 + t0) * L.pitch + j;
    Win2 v;
    if (HK != HK_JACOBI) {
      row_even(c, v.la, v.ma, v.ra);
      row_even(c + XW, v.lb, v.mb, v.rb);
    }
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int i = R0 + t0 + k;
      if (HK != HK_JACOBI) row_even(c + (k + 2) * XW, v.lc, v.mc, v.rc);
      else v.mb = ld2(c + (k + 1) * XW);
      const float2 e = add2(ld2(e1 + k * XW), tapply_H2<HK, IN, false>(L, s, wtab, wi, omega, i, j, v));
      float* d = out + (size_t)k * L.pitch;
      if (IN) {
        st2(d, e);  // e is still read with halos by other CTAs: f is an array of its own
      } else {
        if (inside(i, j, n)) d[0] = e.x;
        if (inside(i, j + 1, n)) d[1] = e.y;
      }
      if (HK != HK_JACOBI) v.shift();
    }
  }
}

template <int HK>
__global__ void __launch_bounds__(NTP, 8) k_upp(const __grid_constant__ UpMaps M, const ProbDev* __restrict__ probs,
                                                ProbState* __restrict__ state, int l, float omega,
                                                const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int ntx = (n + TB - 1) / TB;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float es[UPE_H * XW];  // e, then e1 = e + P e_c in place
  __shared__ __align__(128) float rs[UPR_H * XW];  // r, then t = r - A e1 in place
  __shared__ __align__(128) float ecs[EC_H * EC_W];
  __shared__ float wtab[HK == HK_TABLE ? 9 * MG_PROXY * MG_PROXY : 1];
  __shared__ __align__(8) uint64_t bar;
  const bool in = inner_tile(R0, C0, n);
  float s[9], wi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = L.s[k];
  if (HK == HK_TABLE) load_table(L, in, wtab, wi);
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, ((UPE_H + UPR_H) * XW + EC_H * EC_W) * sizeof(float));
    tma_load_3d(es, &M.e, &bar, C0 - 4, R0 - 2, p);
    tma_load_3d(rs, &M.r, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(ecs, &M.ec, &bar, C0 / 2 - 4, R0 / 2 - 2, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  if (in) upp_tile<HK, true>(L, s, wtab, wi, omega, es, rs, ecs, R0, C0);
  else upp_tile<HK, false>(L, s, wtab, wi, omega, es, rs, ecs, R0, C0);
}

// k_update_residual on constant stencils in pairs (128 threads): the update of the
// iterate over the whole box as 64-bit pairs, then the paired compensated residual of
// k_up0p with b read through L2 (prefetched when the CTA starts).
__global__ void __launch_bounds__(NTP, 8) k_update_residualp(const __grid_constant__ ResMaps X,
                                                             const __grid_constant__ CUtensorMap E,
                                                             const ProbDev* __restrict__ probs,
                                                             ProbState* __restrict__ state, float* __restrict__ partials,
                                                             int ntiles_max, float rtol, int max_cycles,
                                                             float* __restrict__ xhi, float* __restrict__ xlo,
                                                             float* __restrict__ rnew, const float* __restrict__ b0,
                                                             const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[0];
  const int n = L.n;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx;
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float xh[RES_H * XW];
  __shared__ __align__(128) float xl[RES_H * XW];
  __shared__ __align__(128) float es[RES_H * XW];
  __shared__ __align__(8) uint64_t bar;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = L.s[k];
  if (threadIdx.x == 0) tma_prefetch_3d(&X.b, C0, R0, p);
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, 3 * RES_H * XW * sizeof(float));
    tma_load_3d(xh, &X.xh, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(xl, &X.xl, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(es, &E, &bar, C0 - 4, R0 - 1, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  // the box is zero outside the grid in all three arrays, so the update keeps it zero there
  for (int q = 2 * threadIdx.x; q < RES_H * XW; q += 2 * NTP) {
    float2 sum, err, hi, lo;
    two_sum2(ld2(xh + q), ld2(es + q), sum, err);
    err = add2(err, ld2(xl + q));
    fast_two_sum2(sum, err, hi, lo);
    st2(xh + q, hi);
    st2(xl + q, lo);
  }
  __syncthreads();
  const size_t po = (size_t)p * n * L.pitch;
  const float acc = inner_tile(R0, C0, n)
                        ? residual_pair<true>(L, s, xh, xl, R0, C0, rnew + po, xhi + po, xlo + po, b0 + po)
                        : residual_pair<false>(L, s, xh, xl, R0, C0, rnew + po, xhi + po, xlo + po, b0 + po);
  float rhi, rlo;
  if (block_partial_and_last<NTP>(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, rhi, rlo)) {
    if (threadIdx.x == 0) decide(state[p], rhi, rlo, rtol, max_cycles);
  }
}

// -------------------------------------------------------------- pack / unpack
// dense [nprob][n][n] <-> pitched [nprob][n][pitch]; src == nullptr packs zeros
__global__ void k_pack(const float* __restrict__ src, float* __restrict__ dst, int n, int pitch) {
  const int p = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int i = q / n, j = q % n;
  dst[(size_t)p * n * pitch + (size_t)i * pitch + j] = src ? src[(size_t)p * n * n + q] : 0.f;
}

__global__ void k_unpack(const float* __restrict__ src_a, const float* __restrict__ src_b,
                         const ProbState* __restrict__ state, float* __restrict__ dst, int n, int pitch) {
  const int p = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int i = q / n, j = q % n;
  const float* src = (__ldcg(&state[p].cycles) & 1) ? src_b : src_a;
  dst[(size_t)p * n * n + q] = src[(size_t)p * n * pitch + (size_t)i * pitch + j];
}

cudaError_t launch_pack(const float* src, float* dst, int n, int pitch, int nprob, cudaStream_t s) {
  dim3 grid((n * n + 255) / 256, nprob);
  k_pack<<<grid, 256, 0, s>>>(src, dst, n, pitch);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const float* src_a, const float* src_b, const ProbState* state, float* dst, int n, int pitch,
                          int nprob, cudaStream_t s) {
  dim3 grid((n * n + 255) / 256, nprob);
  k_unpack<<<grid, 256, 0, s>>>(src_a, src_b, state, dst, n, pitch);
  return cudaGetLastError();
}

// -------------------------------------------------------------- tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::atomic<void*> fn{nullptr};
  void* f = fn.load(std::memory_order_acquire);
  if (!f) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return nullptr;
    fn.store(f, std::memory_order_release);
  }
  return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
}

// 3-D map {x = n, y = n, z = nprob} over a pitched level array, box bw x bh x 1
void tile_res_box(int* bw, int* bh) {
  *bw = XW;
  *bh = RES_H;
}

bool make_map(CUtensorMap* m, float* base, int n, int pitch, int nprob, int bw, int bh) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)nprob};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float), (cuuint64_t)pitch * n * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool build_tile_maps(TileMaps& T, const LevelArrays& A, int nprob, int lstar, int shape) {
  if (lstar == 0) return true;
  if (shape != MG_SHAPE_TILE32) {
    int bw, bh;
    strip_box(shape, &bw, &bh);
    for (int l = 0; l < lstar; ++l)
      if (!make_map(&T.sr[l], A.r[l], A.n[l], A.pitch[l], nprob, bw, bh)) return false;
    if (!make_map(&T.sr0b, A.r0b, A.n[0], A.pitch[0], nprob, bw, bh)) return false;
  }
  bool ok = make_map(&T.res.xh, A.xh0, A.n[0], A.pitch[0], nprob, XW, RES_H) &&
            make_map(&T.res.xl, A.xl0, A.n[0], A.pitch[0], nprob, XW, RES_H) &&
            make_map(&T.res.b, A.b0, A.n[0], A.pitch[0], nprob, TB, TB);
  for (int l = 0; ok && l < lstar; ++l) {
    ok = make_map(&T.down[l].r, A.r[l], A.n[l], A.pitch[l], nprob, XW, DN_H) &&
         make_map(&T.down[l].e, A.e[l], A.n[l], A.pitch[l], nprob, TB, TB) &&
         make_map(&T.down[l].rc, A.r[l + 1], A.n[l + 1], A.pitch[l + 1], nprob, TC, TC) &&
         make_map(&T.up[l].e, A.e[l], A.n[l], A.pitch[l], nprob, XW, UPE_H) &&
         make_map(&T.up[l].r, A.r[l], A.n[l], A.pitch[l], nprob, XW, UPR_H) &&
         make_map(&T.up[l].ec, l + 1 < lstar ? A.f[l + 1] : A.e[l + 1], A.n[l + 1], A.pitch[l + 1], nprob, EC_W,
                  EC_H);
    if (ok) {
      T.up[l].xh = T.up[l].e;  // the x update is on level 0's fused kernel
      T.up[l].xl = T.up[l].e;
    }
  }
  if (ok) {
    ok = make_map(&T.up0.e, A.e[0], A.n[0], A.pitch[0], nprob, XW, UP0E_H) &&
         make_map(&T.up0.r, A.r[0], A.n[0], A.pitch[0], nprob, XW, UP0R_H) &&
         make_map(&T.up0.ec, 1 < lstar ? A.f[1] : A.e[1], A.n[1], A.pitch[1], nprob, EC_W, EC0_H) &&
         make_map(&T.down0_rb, A.r0b, A.n[0], A.pitch[0], nprob, XW, DN_H) &&
         make_map(&T.up0_rb, A.r0b, A.n[0], A.pitch[0], nprob, XW, UP0R_H);
    T.up0.x = T.res;
    ok = ok && make_map(&T.resb.xh, A.xh0b, A.n[0], A.pitch[0], nprob, XW, RES_H) &&
         make_map(&T.resb.xl, A.xl0b, A.n[0], A.pitch[0], nprob, XW, RES_H);
    T.resb.b = T.res.b;
  }
  return ok;
}

// ---------------------------------------------------------------- launchers
static inline int nlaunch(const CycleArgs& a) { return (a.active && a.nactive > 0) ? a.nactive : a.nprob; }

cudaError_t launch_residual(const CycleArgs& a, float rtol, int max_cycles) {
  const int nt = tiles_per_side(a.n0);
  dim3 grid(nt * nt, nlaunch(a));
  a.prof->launches++;
  a.prof->begin(PK_RESIDUAL, a.stream);
  cudaError_t e;
  if (a.sk == SK_CONST)
    e = launch_pdl(a.pdl, k_residual<SK_CONST>, grid, dim3(NT), 0, a.stream, a.maps->res, (const ProbDev*)a.probs, a.state,
                   a.partials, a.ntiles_max, rtol, max_cycles, a.active);
  else
    e = launch_pdl(a.pdl, k_residual<SK_FIELD>, grid, dim3(NT), 0, a.stream, a.maps->res, (const ProbDev*)a.probs, a.state,
                   a.partials, a.ntiles_max, rtol, max_cycles, a.active);
  a.prof->end(a.stream);
  return e;
}

cudaError_t launch_update_residual(const CycleArgs& a, const CUtensorMap& e0, float rtol, int max_cycles, int parity) {
  const int nt = tiles_per_side(a.n0);
  dim3 grid(nt * nt, nlaunch(a));
  const ResMaps& X = parity ? a.maps->resb : a.maps->res;
  float* rnew = parity ? a.r0a : a.r0b;
  float* xhn = parity ? a.xh0 : a.xh0b;
  float* xln = parity ? a.xl0 : a.xl0b;
  a.prof->launches++;
  a.prof->begin(PK_UP0, a.stream);
  cudaError_t e;
  if (a.sk == SK_CONST)
    e = launch_pdl(a.pdl, k_update_residualp, grid, dim3(NTP), 0, a.stream, X, e0, (const ProbDev*)a.probs, a.state,
                   a.partials, a.ntiles_max, rtol, max_cycles, xhn, xln, rnew, (const float*)a.b0, a.active);
  else
    e = launch_pdl(a.pdl, k_update_residual<SK_FIELD>, grid, dim3(NT), 0, a.stream, X, e0, (const ProbDev*)a.probs,
                   a.state, a.partials, a.ntiles_max, rtol, max_cycles, xhn, xln, rnew, a.active);
  a.prof->end(a.stream);
  return e;
}

// the up-sweep of a tiled level >= 1: the paired kernel on constant stencils, k_up on fields
template <int SK, int HK>
static cudaError_t launch_up(bool pdl, dim3 grid, cudaStream_t s, const UpMaps& um, const ProbDev* probs,
                             ProbState* state, int l, float omega, const int* act) {
  if constexpr (SK == SK_CONST)
    return launch_pdl(pdl, k_upp<HK>, grid, dim3(NTP), 0, s, um, probs, state, l, omega, act);
  else
    return launch_pdl(pdl, k_up<SK, HK, false>, grid, dim3(NT), 0, s, um, probs, state, l, omega, (float*)nullptr,
                      (float*)nullptr, act);
}

// the down-sweep of a tiled level: the paired kernel on constant stencils, k_down on fields
template <int SK, int HK>
static cudaError_t launch_down(bool pdl, dim3 grid, cudaStream_t s, const DownMaps& dm, const ProbDev* probs,
                               ProbState* state, int l, float omega, const int* act) {
  if constexpr (SK == SK_CONST) {
    // two tiles per CTA once the launch is several waves deep (8 CTAs per SM)
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int tpc = (long long)grid.x * grid.y >= 4ll * 8 * (nsm > 0 ? nsm : 1) ? 2 : 1;
    const dim3 g((grid.x + tpc - 1) / tpc, grid.y);
    return launch_pdl(pdl, k_downp<HK>, g, dim3(NTP), 0, s, dm, probs, state, l, omega, tpc, act);
  }
  else
    return launch_pdl(pdl, k_down<SK, HK>, grid, dim3(NT), 0, s, dm, probs, state, l, omega, act);
}

// level 0 of the up-sweep: the paired kernel on constant stencils, k_up0 on per-point fields
template <int SK, int HK>
static cudaError_t launch_up0(bool pdl, dim3 grid, cudaStream_t s, const Up0Maps& um, const ProbDev* probs,
                              ProbState* state, float* partials, int ntiles_max, float omega, float rtol,
                              int max_cycles, float* xhn, float* xln, float* rnew, const float* b0, const int* act) {
  if constexpr (SK == SK_CONST)
    return launch_pdl(pdl, k_up0p<HK>, grid, dim3(NTP), 0, s, um, probs, state, partials, ntiles_max, omega, rtol,
                      max_cycles, xhn, xln, rnew, b0, act);
  else
    return launch_pdl(pdl, k_up0<SK, HK>, grid, dim3(NT), 0, s, um, probs, state, partials, ntiles_max, omega, rtol,
                      max_cycles, xhn, xln, rnew, b0, act);
}

cudaError_t launch_cycle(const CycleArgs& a, float rtol, int max_cycles, int parity) {
  if (a.generic) return launch_cycle_linear(a, rtol, max_cycles, parity);
  // the fused tile kernels exist for Jacobi and per-point 3x3 kernels only
  if (a.hk != HK_JACOBI && a.hk != HK_TABLE && a.hk != HK_FIELD) return cudaErrorNotSupported;
  const int ls = a.lstar, np = nlaunch(a);
  const ProbDev* probs = a.probs;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < ls && e == cudaSuccess; ++l) {
    const int nt = tiles_per_side(a.nl[l]);
    dim3 grid(nt * nt, np);
    a.prof->launches++;
    a.prof->begin(l == 0 ? PK_DOWN0 : PK_DOWN, a.stream);
    if (a.shape == MG_SHAPE_PSTRIP ? pdown_applies(a, l, np) : a.shape != MG_SHAPE_TILE32) {
      e = launch_sdown(a, (l == 0 && parity) ? a.maps->sr0b : a.maps->sr[l], l, np);
    } else {
      DownMaps dm = a.maps->down[l];
      if (l == 0 && parity) dm.r = a.maps->down0_rb;
      MG_DISPATCH(a.sk, a.hk, (e = launch_down<SK_, HK_>(a.pdl, grid, a.stream, dm, probs, a.state, l, a.omega, a.active)));
    }
    a.prof->end(a.stream);
  }
  if (e != cudaSuccess) return e;
  e = launch_tail(a);
  for (int l = ls - 1; l >= 0 && e == cudaSuccess; --l) {
    const int nt = tiles_per_side(a.nl[l]);
    dim3 grid(nt * nt, np);
    // The kernel after the cluster tail waits for it by plain stream order: with
    // programmatic serialisation the cycle measured no faster (the tail's clusters hold
    // whole SMs, so the next kernel has little room to start early).
    const bool pdl = a.pdl && !(a.ctail && l == ls - 1);
    a.prof->launches++;
    a.prof->begin(l == 0 ? PK_UP0 : PK_UP, a.stream);
    if (l == 0) {
      Up0Maps um = a.maps->up0;
      if (parity) {
        um.r = a.maps->up0_rb;
        um.x = a.maps->resb;
      }
      float* rnew = parity ? a.r0a : a.r0b;
      float* xhn = parity ? a.xh0 : a.xh0b;
      float* xln = parity ? a.xl0 : a.xl0b;
      MG_DISPATCH(a.sk, a.hk,
                  (e = launch_up0<SK_, HK_>(pdl, grid, a.stream, um, probs, a.state, a.partials, a.ntiles_max, a.omega,
                                            rtol, max_cycles, xhn, xln, rnew, a.b0, a.active)));
    }
    else
      MG_DISPATCH(a.sk, a.hk, (e = launch_up<SK_, HK_>(pdl, grid, a.stream, a.maps->up[l], probs, a.state, l, a.omega,
                                                       a.active)));
    a.prof->end(a.stream);
  }
  return e;
}

}  // namespace mg
