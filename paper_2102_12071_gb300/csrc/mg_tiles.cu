// mg_tiles.cu -- the tiled level kernels of the batched V-cycle (levels n_l > MG_TAIL_N).
//
// Each CTA owns a 32 x 32 block of fine points of one problem.  All its inputs, halos
// included, arrive as TMA bulk tensor copies issued by one thread into shared memory
// (one mbarrier per CTA); the copy engine zero-fills everything outside the grid, which is
// exactly the homogeneous Dirichlet exterior.  Level vectors use a row pitch that is a
// multiple of 32 floats (128-byte rows) and all problems of a level are one 3-D tensor
// {x, y, problem}, so one tensor map serves the whole batch.
//   k_residual  r = b - A (x_hi + x_lo), compensated (float-float), ||r||^2, stopping test
//   k_down(l)   e = H r, s = r - A e, r_{l+1} = P^T s         (Algorithm 1, pre-smoothing and restriction)
//   k_up(l)     e1 = e + P e_{l+1}, e = e1 + H (r - A e1)      (Algorithm 1, correction and post-smoothing);
//               on level 0 the correction is added to the float-float iterate.
#include <cudaTypedefs.h>

#include <atomic>

#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_ops.cuh"
#include "mg_reduce.cuh"
#include "mg_tma.cuh"

namespace mg {

constexpr int TB = 32;           // fine tile side
constexpr int NT = 256;          // threads per CTA (8 warps)
constexpr int NW = NT / 32;
constexpr int XW = TB + 8;       // box width: columns C0-4 .. C0+35 (x start 16-byte aligned)
constexpr int RES_H = TB + 2;    // k_residual x boxes: rows R0-1 .. R0+32
constexpr int DN_H = TB + 5;     // k_down r box: rows R0-2 .. R0+34
constexpr int UPE_H = TB + 4;    // k_up e box: rows R0-2 .. R0+33
constexpr int UPR_H = TB + 2;    // k_up r box: rows R0-1 .. R0+32
constexpr int EC_W = TB / 2 + 8; // k_up coarse box: columns C0/2-4 .. C0/2+19
constexpr int EC_H = TB / 2 + 3; //                  rows    R0/2-2 .. R0/2+16
constexpr int ES_DN = TB + 3;    // k_down e buffer side (rows/cols R0-1 .. R0+33)

template <int SK>
__device__ __forceinline__ void load_stencil_t(const LevelDev& L, float (&s)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
}

// Network kernels of a constant-stencil level for one tile.  If every point within two
// of the tile is at least MG_NET_MARGIN from the edges, all of them use the interior class
// and the 9 taps go to registers; otherwise the whole class table is copied to shared
// memory.  Returns true for the interior case (uniform over the CTA).
__device__ __forceinline__ bool load_table(const LevelDev& L, int R0, int C0, float* wtab, float (&wi)[9]) {
  const int n = L.n, T = L.T, M = MG_NET_MARGIN;
  const bool interior = T == MG_PROXY && R0 - 2 >= M && R0 + TB + 2 <= n - 1 - M && C0 - 2 >= M &&
                        C0 + TB + 2 <= n - 1 - M;
  if (interior) {
#pragma unroll
    for (int k = 0; k < 9; ++k) wi[k] = L.W[k * T * T + M * T + M];
  } else {
    const int cnt = 9 * T * T;
    for (int t = threadIdx.x; t < cnt; t += NT) wtab[t] = L.W[t];
  }
  return interior;
}

// H v at (i, j): the interior kernel from registers when the tile is interior
template <int SK, int HK>
__device__ __forceinline__ float smooth_at(const LevelDev& L, const float (&s)[9], const float* wtab,
                                           const float (&wi)[9], bool interior, float omega, int i, int j,
                                           const float* c, int ts) {
  if (HK == HK_TABLE && interior) {
    float acc = wi[4] * c[0];
    acc = fmaf(wi[0], c[-ts - 1], acc);
    acc = fmaf(wi[1], c[-ts], acc);
    acc = fmaf(wi[2], c[-ts + 1], acc);
    acc = fmaf(wi[3], c[-1], acc);
    acc = fmaf(wi[5], c[1], acc);
    acc = fmaf(wi[6], c[ts - 1], acc);
    acc = fmaf(wi[7], c[ts], acc);
    acc = fmaf(wi[8], c[ts + 1], acc);
    return acc;
  }
  return smoother_apply<SK, HK>(L, s, wtab, omega, i, j, c, ts);
}

// Waits for the CTA's copies; on expiry marks the problem timed out (status 4) and waits
// once more, bounded, for copies still in flight.  Returns false in every thread then.
__device__ __forceinline__ bool tile_wait(uint64_t* bar, ProbState& st) {
  const bool ok = mbar_wait(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      st.status = 4;
      st.active = 0;
    }
    mbar_wait(bar, 0);
    return false;
  }
  return true;
}

// ------------------------------------------------------------------ k_residual
template <int SK>
__global__ void __launch_bounds__(NT) k_residual(const __grid_constant__ ResMaps M, const ProbDev* __restrict__ probs,
                                                 ProbState* __restrict__ state, float* __restrict__ partials,
                                                 int ntiles_max, float rtol, int max_cycles,
                                                 const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[0];
  const int n = L.n, pitch = L.pitch;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx;
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float XH[RES_H * XW];
  __shared__ __align__(128) float XL[RES_H * XW];
  __shared__ __align__(128) float BB[TB * TB];
  __shared__ __align__(8) uint64_t bar;
  float s[9];
  load_stencil_t<SK>(L, s);
  pdl_wait();
  if (!state[p].active) return;
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
  const size_t nn = (size_t)n * n;
  float acc = 0.f;
  const int tx = threadIdx.x & 31;
  for (int ty = threadIdx.x >> 5; ty < TB; ty += NW) {
    const int i = R0 + ty, j = C0 + tx;
    if (!in_grid(i, j, n)) continue;
    const int c = (ty + 1) * XW + tx + 4;
    float hi = BB[ty * TB + tx], lo = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int off = (k / 3 - 1) * XW + (k % 3 - 1);
      const float a = (SK == SK_CONST) ? s[k] : __ldg(L.st + k * nn + (size_t)i * n + j);
      const float x = XH[c + off];
      const float pr = a * x;
      const float pe = fmaf(a, x, -pr);
      float sum, err;
      two_sum(hi, -pr, sum, err);
      hi = sum;
      lo += err - pe;
      lo = fmaf(-a, XL[c + off], lo);
    }
    const float r = hi + lo;
    L.r[(size_t)i * pitch + j] = r;
    acc = fmaf(r, r, acc);
  }
  float rhi, rlo;
  if (block_partial_and_last<NT>(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, rhi, rlo)) {
    if (threadIdx.x == 0) decide(state[p], rhi, rlo, rtol, max_cycles);
  }
}

// ---------------------------------------------------------------------- k_down
template <int SK, int HK>
__global__ void __launch_bounds__(NT) k_down(const __grid_constant__ CUtensorMap mr, const ProbDev* __restrict__ probs,
                                             ProbState* __restrict__ state, int l, float omega,
                                             const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const LevelDev Lc = probs[p].lv[l + 1];
  const int n = L.n, nc = Lc.n, pitch = L.pitch, cpitch = Lc.pitch;
  const int ntx = (n + TB - 1) / TB;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float rs[DN_H * XW];  // r, then s = r - A e in place
  __shared__ float es[ES_DN * ES_DN];
  __shared__ float wtab[9 * MG_PROXY * MG_PROXY];
  __shared__ __align__(8) uint64_t bar;
  float s[9], wi[9];
  load_stencil_t<SK>(L, s);
  bool interior = false;
  if (HK == HK_TABLE) interior = load_table(L, R0, C0, wtab, wi);
  pdl_wait();
  if (!state[p].active) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, DN_H * XW * sizeof(float));
    tma_load_3d(rs, &mr, &bar, C0 - 4, R0 - 2, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  // pre-smoothing from zero: e = H r on rows/cols R0-1 .. R0+33
  for (int t = threadIdx.x; t < ES_DN * ES_DN; t += NT) {
      const int ti = t / ES_DN, tj = t - ti * ES_DN;
      const int i = R0 - 1 + ti, j = C0 - 1 + tj;
      float v = 0.f;
      if (in_grid(i, j, n)) {
        v = smooth_at<SK, HK>(L, s, wtab, wi, interior, omega, i, j, rs + (ti + 1) * XW + tj + 3, XW);
        if (ti >= 1 && ti <= TB && tj >= 1 && tj <= TB) L.e[(size_t)i * pitch + j] = v;
      }
      es[ti * ES_DN + tj] = v;
    }
  __syncthreads();
  // s = r - A e on rows/cols R0 .. R0+32, written over r
  for (int t = threadIdx.x; t < (TB + 1) * (TB + 1); t += NT) {
      const int ti = t / (TB + 1), tj = t - ti * (TB + 1);
      const int i = R0 + ti, j = C0 + tj;
      float* rp = rs + (ti + 2) * XW + tj + 4;
      float v = 0.f;
      if (in_grid(i, j, n)) v = *rp - stencil_apply<SK>(L, s, i, j, es + (ti + 1) * ES_DN + tj + 1, ES_DN);
      *rp = v;
    }
  __syncthreads();
  // r_c = P^T s for the 16 x 16 coarse points centred in the tile
  {
    const int a = threadIdx.x >> 4, b = threadIdx.x & 15;
    const int I = R0 / 2 + a, J = C0 / 2 + b;
    if (I < nc && J < nc) Lc.r[(size_t)I * cpitch + J] = restrict_at(rs + (2 * a + 3) * XW + 2 * b + 5, XW);
  }
}

// ------------------------------------------------------------------------ k_up
template <int SK, int HK, bool UPDX>
__global__ void __launch_bounds__(NT) k_up(const __grid_constant__ UpMaps M, const ProbDev* __restrict__ probs,
                                           ProbState* __restrict__ state, int l, float omega, float* __restrict__ xhi,
                                           float* __restrict__ xlo, const int* __restrict__ act) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, nc = probs[p].lv[l + 1].n, pitch = L.pitch;
  const int ntx = (n + TB - 1) / TB;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  __shared__ __align__(128) float es[UPE_H * XW];   // e, then e1 = e + P e_c in place
  __shared__ __align__(128) float rs[UPR_H * XW];   // r, then t = r - A e1 in place
  __shared__ __align__(128) float ecs[EC_H * EC_W];
  __shared__ __align__(128) float xhs[UPDX ? TB * TB : 4];
  __shared__ __align__(128) float xls[UPDX ? TB * TB : 4];
  __shared__ float wtab[9 * MG_PROXY * MG_PROXY];
  __shared__ __align__(8) uint64_t bar;
  const int I0 = R0 / 2 - 2, J0 = C0 / 2 - 4;
  float s[9], wi[9];
  load_stencil_t<SK>(L, s);
  bool interior = false;
  if (HK == HK_TABLE) interior = load_table(L, R0, C0, wtab, wi);
  pdl_wait();
  if (!state[p].active) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, ((UPE_H + UPR_H) * XW + EC_H * EC_W + (UPDX ? 2 * TB * TB : 0)) * sizeof(float));
    tma_load_3d(es, &M.e, &bar, C0 - 4, R0 - 2, p);
    tma_load_3d(rs, &M.r, &bar, C0 - 4, R0 - 1, p);
    tma_load_3d(ecs, &M.ec, &bar, J0, I0, p);
    if (UPDX) {
      tma_load_3d(xhs, &M.xh, &bar, C0, R0, p);
      tma_load_3d(xls, &M.xl, &bar, C0, R0, p);
    }
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  (void)nc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // e1 = e + P e_c on rows/cols R0-2 .. R0+33 (zero outside the grid)
  for (int t = threadIdx.x; t < (TB + 4) * (TB + 4); t += NT) {
      const int ti = t / (TB + 4), tj = t - ti * (TB + 4);
      const int i = R0 - 2 + ti, j = C0 - 2 + tj;
      float* ep = es + ti * XW + tj + 2;
      *ep = in_grid(i, j, n) ? *ep + prolong_at(i, j, ecs, I0, J0, EC_W) : 0.f;
    }
  __syncthreads();
  // t = r - A e1 on rows/cols R0-1 .. R0+32
  for (int t = threadIdx.x; t < (TB + 2) * (TB + 2); t += NT) {
      const int ti = t / (TB + 2), tj = t - ti * (TB + 2);
      const int i = R0 - 1 + ti, j = C0 - 1 + tj;
      float* rp = rs + ti * XW + tj + 3;
      *rp = in_grid(i, j, n) ? *rp - stencil_apply<SK>(L, s, i, j, es + (ti + 1) * XW + tj + 3, XW) : 0.f;
    }
  __syncthreads();
  // post-smoothing on the owned points: e = e1 + H t
  const int tx = lane;
  for (int ty = warp; ty < TB; ty += NW) {
    const int i = R0 + ty, j = C0 + tx;
    if (!in_grid(i, j, n)) continue;
    const float e = es[(ty + 2) * XW + tx + 4] +
                    smooth_at<SK, HK>(L, s, wtab, wi, interior, omega, i, j, rs + (ty + 1) * XW + tx + 4, XW);
    const size_t g = (size_t)p * n * pitch + (size_t)i * pitch + j;
    if (UPDX) {
      float hi = xhs[ty * TB + tx], lo = xls[ty * TB + tx], sum, err;
      two_sum(hi, e, sum, err);
      err += lo;
      fast_two_sum(sum, err, hi, lo);
      xhi[g] = hi;
      xlo[g] = lo;
    } else {
      L.e[(size_t)i * pitch + j] = e;
    }
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

__global__ void k_unpack(const float* __restrict__ src, float* __restrict__ dst, int n, int pitch) {
  const int p = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int i = q / n, j = q % n;
  dst[(size_t)p * n * n + q] = src[(size_t)p * n * pitch + (size_t)i * pitch + j];
}

cudaError_t launch_pack(const float* src, float* dst, int n, int pitch, int nprob, cudaStream_t s) {
  dim3 grid((n * n + 255) / 256, nprob);
  k_pack<<<grid, 256, 0, s>>>(src, dst, n, pitch);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const float* src, float* dst, int n, int pitch, int nprob, cudaStream_t s) {
  dim3 grid((n * n + 255) / 256, nprob);
  k_unpack<<<grid, 256, 0, s>>>(src, dst, n, pitch);
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
static bool make_map(CUtensorMap* m, float* base, int n, int pitch, int nprob, int bw, int bh) {
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

bool build_tile_maps(TileMaps& T, const LevelArrays& A, int nprob, int lstar) {
  if (lstar == 0) return true;
  bool ok = make_map(&T.res.xh, A.xh0, A.n[0], A.pitch[0], nprob, XW, RES_H) &&
            make_map(&T.res.xl, A.xl0, A.n[0], A.pitch[0], nprob, XW, RES_H) &&
            make_map(&T.res.b, A.b0, A.n[0], A.pitch[0], nprob, TB, TB);
  for (int l = 0; ok && l < lstar; ++l) {
    ok = make_map(&T.down[l], A.r[l], A.n[l], A.pitch[l], nprob, XW, DN_H) &&
         make_map(&T.up[l].e, A.e[l], A.n[l], A.pitch[l], nprob, XW, UPE_H) &&
         make_map(&T.up[l].r, A.r[l], A.n[l], A.pitch[l], nprob, XW, UPR_H) &&
         make_map(&T.up[l].ec, A.e[l + 1], A.n[l + 1], A.pitch[l + 1], nprob, EC_W, EC_H);
    if (ok && l == 0)
      ok = make_map(&T.up[0].xh, A.xh0, A.n[0], A.pitch[0], nprob, TB, TB) &&
           make_map(&T.up[0].xl, A.xl0, A.n[0], A.pitch[0], nprob, TB, TB);
    else if (ok) {
      T.up[l].xh = T.up[l].e;  // unused on levels >= 1
      T.up[l].xl = T.up[l].e;
    }
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

cudaError_t launch_cycle(const CycleArgs& a) {
  const int ls = a.lstar, np = nlaunch(a);
  const ProbDev* probs = a.probs;
  float* const nul = nullptr;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < ls && e == cudaSuccess; ++l) {
    const int nt = tiles_per_side(a.nl[l]);
    dim3 grid(nt * nt, np);
    a.prof->launches++;
    a.prof->begin(l == 0 ? PK_DOWN0 : PK_DOWN, a.stream);
    MG_DISPATCH(a.sk, a.hk,
                (e = launch_pdl(a.pdl, k_down<SK_, HK_>, grid, dim3(NT), 0, a.stream, a.maps->down[l], probs, a.state, l,
                                a.omega, a.active)));
    a.prof->end(a.stream);
  }
  if (e != cudaSuccess) return e;
  e = launch_tail(a);
  for (int l = ls - 1; l >= 0 && e == cudaSuccess; --l) {
    const int nt = tiles_per_side(a.nl[l]);
    dim3 grid(nt * nt, np);
    a.prof->launches++;
    a.prof->begin(l == 0 ? PK_UP0 : PK_UP, a.stream);
    if (l == 0)
      MG_DISPATCH(a.sk, a.hk,
                  (e = launch_pdl(a.pdl, k_up<SK_, HK_, true>, grid, dim3(NT), 0, a.stream, a.maps->up[0], probs, a.state, 0,
                                  a.omega, a.xh0, a.xl0, a.active)));
    else
      MG_DISPATCH(a.sk, a.hk,
                  (e = launch_pdl(a.pdl, k_up<SK_, HK_, false>, grid, dim3(NT), 0, a.stream, a.maps->up[l], probs, a.state,
                                  l, a.omega, nul, nul, a.active)));
    a.prof->end(a.stream);
  }
  return e;
}

}  // namespace mg
