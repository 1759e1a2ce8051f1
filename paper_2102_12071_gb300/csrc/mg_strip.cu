// mg_strip.cu -- the tiled levels of the batched V-cycle laid out in warp strips.
//
// A warp owns 26 consecutive columns of a level and walks down the rows of its CTA's
// block; lane k holds column c0 - 2 + k (c0 the first owned column), so the lanes at
// either end carry the halo columns the stencil, smoother and restriction need.  The
// horizontal neighbours of a value come from the adjacent lanes by warp shuffles and the
// vertical ones from the rows the warp has already walked, held in registers: a point
// costs one shared-memory load of each input array instead of a 3x3 window per pass.
// A CTA of WPC warps owns WPC * 26 columns and H rows; its input block with halos arrives
// as one TMA bulk tensor copy (zero-filled outside the grid: the Dirichlet exterior).
//   k_sdown(l)  e = H r, s = r - A e, r_{l+1} = P^T s   (Algorithm 1, pre-smoothing and restriction)
#include <cudaTypedefs.h>

#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_tile.cuh"
#include "mg_tma.cuh"

namespace mg {

constexpr int SW = 26;  // owned columns per warp

template <int WPC, int H>
struct Strip {
  static constexpr int NT = 32 * WPC;  // threads per CTA
  static constexpr int CW = SW * WPC;  // owned columns per CTA
  static constexpr int BW = CW + 8;    // box columns C0-4 .. C0+CW+3 (x start 16-byte aligned)
  static constexpr int BH = H + 5;     // box rows R0-2 .. R0+H+2
  // resident CTAs per SM the register bound aims at (shared memory allows as many): about
  // 40 warps per SM on 32-row blocks, 24 on 64-row blocks
  static constexpr int MINB = H == 32 ? 40 / WPC : 3;
  static_assert(H % 2 == 0, "coarse rows need an even first row");
  static_assert(BW <= 256 && BH <= 256, "TMA box limit");
};

// the value of the lanes to the left and to the right (lanes 0 and 31 get their own)
struct Row3 {
  float l, c, r;
};
__device__ __forceinline__ Row3 row3(float c) {
  Row3 v;
  v.c = c;
  v.l = __shfl_up_sync(0xffffffffu, c, 1);
  v.r = __shfl_down_sync(0xffffffffu, c, 1);
  return v;
}

// sum over the 3x3 neighbourhood (rows a = i-1, b = i, c = i+1), centre first
__device__ __forceinline__ float dot9r(const float (&w)[9], const Row3& a, const Row3& b, const Row3& c) {
  float acc = w[4] * b.c;
  acc = fmaf(w[0], a.l, acc);
  acc = fmaf(w[1], a.c, acc);
  acc = fmaf(w[2], a.r, acc);
  acc = fmaf(w[3], b.l, acc);
  acc = fmaf(w[5], b.r, acc);
  acc = fmaf(w[6], c.l, acc);
  acc = fmaf(w[7], c.c, acc);
  acc = fmaf(w[8], c.r, acc);
  return acc;
}

// stencil of point (i, j): the level's constant one, or the per-point field
template <int SK>
__device__ __forceinline__ void stencil_at(const LevelDev& L, const float (&s)[9], int i, int j, float (&a)[9]) {
  if (SK == SK_CONST) {
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = s[k];
  } else {
    const size_t nn = (size_t)L.n * L.n;
    const float* p = L.st + (size_t)i * L.n + j;
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = __ldg(p + k * nn);
  }
}

// H v at (i, j), a point inside the grid.  Jacobi: (omega / D) v; table: the interior
// kernel wi unless the point lies within MG_NET_MARGIN of an edge (its class from the
// level's table); field: the point's own kernel.
template <int SK, int HK>
__device__ __forceinline__ float strip_H(const LevelDev& L, const float (&s)[9], const float (&wi)[9], float omega,
                                         int i, int j, bool margin, const Row3& a, const Row3& b, const Row3& c) {
  if (HK == HK_JACOBI) {
    const float d = (SK == SK_CONST) ? s[4] : __ldg(L.st + 4 * (size_t)L.n * L.n + (size_t)i * L.n + j);
    return (omega / d) * b.c;
  }
  if (HK == HK_TABLE) {
    if (!margin) return dot9r(wi, a, b, c);
    const int T = L.T;
    const float* p = L.W + kclass(i, L.n, T) * T + kclass(j, L.n, T);
    float w[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = __ldg(p + k * T * T);
    return dot9r(w, a, b, c);
  }
  const size_t nn = (size_t)L.n * L.n;
  const float* p = L.W + (size_t)i * L.n + j;
  float w[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = __ldg(p + k * nn);
  return dot9r(w, a, b, c);
}

// ---------------------------------------------------------------------- k_sdown
// Box row q holds grid row R0 - 2 + q.  Walking q = 0 .. BH-1, the warp forms e = H r on
// box row q-1 (grid rows R0-1 .. R0+H+1), s = r - A e on box row q-2 (R0 .. R0+H) and the
// column sums v = s/2 + s + s/2 of the restriction over fine rows 2I+2, 2I+3, 2I+4 of box
// coordinates; at each coarse row it finishes P^T s with the row sums of the neighbouring
// lanes.  Correct values: e on lanes 1..30, s on 2..29, r_c on the odd lanes 3..27.
template <int SK, int HK, int WPC, int H>
__global__ void __launch_bounds__(32 * WPC, Strip<WPC, H>::MINB) k_sdown(const __grid_constant__ CUtensorMap Mr,
                                                    const ProbDev* __restrict__ probs, ProbState* __restrict__ state,
                                                    int l, float omega, const int* __restrict__ act) {
  using G = Strip<WPC, H>;
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int ncx = (n + G::CW - 1) / G::CW, ncy = (n + H - 1) / H;
  if ((int)blockIdx.x >= ncx * ncy) return;
  const int R0 = ((int)blockIdx.x / ncx) * H, C0 = ((int)blockIdx.x % ncx) * G::CW;
  __shared__ __align__(128) float rs[G::BH * G::BW];
  __shared__ __align__(8) uint64_t bar;
  float s[9], wi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  if (HK == HK_TABLE) {
    const int T = L.T, M = MG_NET_MARGIN;
#pragma unroll
    for (int k = 0; k < 9; ++k) wi[k] = T == MG_PROXY ? L.W[k * T * T + M * T + M] : 0.f;
  }
  float* const rc_out = probs[p].lv[l + 1].r;  // per-problem pitched arrays
  const int nc = probs[p].lv[l + 1].n, pc = probs[p].lv[l + 1].pitch, pitch = L.pitch;
  float* const e_out = L.e;
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, G::BH * G::BW * sizeof(float));
    tma_load_3d(rs, &Mr, &bar, C0 - 4, R0 - 2, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c0 = C0 + SW * w;            // first owned column of the warp
  const int j = c0 - 2 + lane;           // this lane's column
  const bool jin = (unsigned)j < (unsigned)n;
  const bool own = lane >= 2 && lane < 2 + SW && jin;
  // points within MG_NET_MARGIN of the left or right edge take their kernel from the table
  const bool jmargin = HK == HK_TABLE && (L.T != MG_PROXY || j < MG_NET_MARGIN || j >= n - MG_NET_MARGIN);
  const float* col = rs + SW * w + 2 + lane;
  // coarse output of the odd lanes 3 .. 27: column c0/2 + (lane - 3)/2
  const int Jc = (c0 >> 1) + ((lane - 3) >> 1);
  const bool cown = (lane & 1) && lane >= 3 && lane <= 27 && Jc < nc;

  Row3 ra = row3(col[0]), rb = row3(col[G::BW]);  // r on box rows q-2, q-1
  Row3 ea, eb;                                     // e on box rows q-3, q-2
  ea.l = ea.c = ea.r = 0.f;
  eb = ea;
  float v = 0.f;                                   // column sum of the current coarse row
#pragma unroll
  for (int q = 2; q < G::BH; ++q) {
    const Row3 rc = row3(col[q * G::BW]);
    // e on box row q-1 = grid row ie
    const int ie = R0 + q - 3;
    float e = 0.f;
    if (jin && (unsigned)ie < (unsigned)n) {
      const bool margin = HK == HK_TABLE && (jmargin || ie < MG_NET_MARGIN || ie >= n - MG_NET_MARGIN);
      e = strip_H<SK, HK>(L, s, wi, omega, ie, j, margin, ra, rb, rc);
    }
    const Row3 ec = row3(e);
    if (q >= 3 && q < H + 3 && own && ie < n) e_out[(size_t)ie * pitch + j] = e;
    if (q >= 4) {
      // s on box row q-2 = grid row is (needed inside the grid only)
      const int is = R0 + q - 4;
      float sv = 0.f;
      if (jin && is < n) {
        float a[9];
        stencil_at<SK>(L, s, is, j, a);
        sv = ra.c - dot9r(a, ea, eb, ec);
      }
      // restriction: box row qs = q-2 is fine row 2I+2 (even: ends coarse row I-1, starts
      // I) or 2I+3 (odd: centre of I) of the CTA's coarse rows I = 0 .. H/2-1
      const int qs = q - 2;
      if ((qs & 1) == 0) {
        if (qs >= 4) {
          v = fmaf(0.5f, sv, v);
          const float rcv = fmaf(0.5f, __shfl_up_sync(0xffffffffu, v, 1) + __shfl_down_sync(0xffffffffu, v, 1), v);
          const int Ic = (R0 >> 1) + (qs - 4) / 2;
          if (cown && Ic < nc) rc_out[(size_t)Ic * pc + Jc] = rcv;
        }
        v = 0.5f * sv;
      } else {
        v += sv;
      }
    }
    ra = rb;
    rb = rc;
    ea = eb;
    eb = ec;
  }
}

// ---------------------------------------------------------------- launchers
template <int WPC, int H>
static cudaError_t sdown_shape(const CycleArgs& a, const CUtensorMap& m, int l, dim3 grid) {
  using G = Strip<WPC, H>;
  cudaError_t e = cudaSuccess;
  MG_DISPATCH(a.sk, a.hk,
              (e = launch_pdl(a.pdl, k_sdown<SK_, HK_, WPC, H>, grid, dim3(G::NT), 0, a.stream, m,
                              (const ProbDev*)a.probs, a.state, l, a.omega, a.active)));
  return e;
}

void strip_box(int shape, int* bw, int* bh) {
  switch (shape) {
    case MG_SHAPE_STRIP4x32: *bw = Strip<4, 32>::BW; *bh = Strip<4, 32>::BH; return;
    case MG_SHAPE_STRIP8x64: *bw = Strip<8, 64>::BW; *bh = Strip<8, 64>::BH; return;
    default: *bw = Strip<8, 32>::BW; *bh = Strip<8, 32>::BH; return;
  }
}

static void strip_cta(int shape, int* cw, int* h) {
  switch (shape) {
    case MG_SHAPE_STRIP4x32: *cw = Strip<4, 32>::CW; *h = 32; return;
    case MG_SHAPE_STRIP8x64: *cw = Strip<8, 64>::CW; *h = 64; return;
    default: *cw = Strip<8, 32>::CW; *h = 32; return;
  }
}

cudaError_t launch_sdown(const CycleArgs& a, const CUtensorMap& m, int l, int np) {
  int cw, h;
  strip_cta(a.shape, &cw, &h);
  const int n = a.nl[l];
  const dim3 grid(((n + cw - 1) / cw) * ((n + h - 1) / h), np);
  switch (a.shape) {
    case MG_SHAPE_STRIP4x32: return sdown_shape<4, 32>(a, m, l, grid);
    case MG_SHAPE_STRIP8x64: return sdown_shape<8, 64>(a, m, l, grid);
    default: return sdown_shape<8, 32>(a, m, l, grid);
  }
}

}  // namespace mg
