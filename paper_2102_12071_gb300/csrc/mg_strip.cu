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
#include "mg_reduce.cuh"
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
  // 32 warps per SM on 32-row blocks, 24 on 64-row blocks
  static constexpr int MINB = H == 32 ? 32 / WPC : 3;
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
// Box row q holds grid row R0 - 2 + q.  Walking q = 2 .. BH-1, the warp forms e = H r on
// box row q-1 (grid rows R0-1 .. R0+H+1), s = r - A e on box row q-2 (R0 .. R0+H) and the
// column sums v = s/2 + s + s/2 of the restriction over fine rows 2I+2, 2I+3, 2I+4 of box
// coordinates; at each coarse row it finishes P^T s with the row sums of the neighbouring
// lanes.  Correct values: e on lanes 1..30, s on 2..29, r_c on the odd lanes 3..27.
// The walk is a loop over chunks of six rows (the periods of the three-row windows and of
// the restriction's row parity), so the register windows rotate without copies while the
// code stays small enough for the instruction cache.  EDGE selects the variant for warps
// that touch the boundary: bounds checks, and class-table kernels within MG_NET_MARGIN of
// an edge; warps away from it run without either.
struct DownCtx {
  float s[9], wi[9];
  float omega;
  int n, R0, j, nc, pitch, pc, Jc;
  bool jin, own, cown, jmargin;
  const float* col;
  float* e_out;
  float* rc_out;
};

template <int SK, int HK, int H, int BW, bool EDGE>
__device__ __forceinline__ void sdown_walk(const LevelDev& L, const DownCtx& c) {
  constexpr int BH = H + 5;
  Row3 ra = row3(c.col[0]), rb = row3(c.col[BW]);  // r on box rows q-2, q-1
  Row3 ea, eb;                                       // e on box rows q-3, q-2
  ea.l = ea.c = ea.r = 0.f;
  eb = ea;
  float v = 0.f;  // column sum of the current coarse row
#pragma unroll 1
  for (int q0 = 2; q0 < BH; q0 += 6) {
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int q = q0 + u;
      if (q < BH) {
        const Row3 rc = row3(c.col[q * BW]);
        const int ie = c.R0 + q - 3;  // e on box row q-1
        float e = 0.f;
        if (!EDGE || (c.jin && (unsigned)ie < (unsigned)c.n)) {
          const bool margin = EDGE && (c.jmargin || ie < MG_NET_MARGIN || ie >= c.n - MG_NET_MARGIN);
          e = strip_H<SK, HK>(L, c.s, c.wi, c.omega, ie, c.j, margin, ra, rb, rc);
        }
        const Row3 ec = row3(e);
        if (q >= 3 && q < H + 3 && c.own && (!EDGE || ie < c.n)) __stcg(c.e_out + (size_t)ie * c.pitch + c.j, e);
        if (q >= 4) {
          const int is = c.R0 + q - 4;  // s on box row q-2 (needed inside the grid only)
          float sv = 0.f;
          if (!EDGE || (c.jin && is < c.n)) {
            float a[9];
            stencil_at<SK>(L, c.s, is, c.j, a);
            sv = ra.c - dot9r(a, ea, eb, ec);
          }
          // box row qs = q-2 is fine row 2I+2 (even: ends coarse row I-1, starts I) or 2I+3
          // (odd: centre of I) of the CTA's coarse rows I = 0 .. H/2-1; q0 - 2 is a
          // multiple of 6, so the parity of qs is that of u
          const int qs = q - 2;
          if ((u & 1) == 0) {
            if (qs >= 4) {
              v = fmaf(0.5f, sv, v);
              const float rcv = fmaf(0.5f, __shfl_up_sync(0xffffffffu, v, 1) + __shfl_down_sync(0xffffffffu, v, 1), v);
              const int Ic = (c.R0 >> 1) + ((qs - 4) >> 1);
              if (c.cown && (!EDGE || Ic < c.nc)) __stcg(c.rc_out + (size_t)Ic * c.pc + c.Jc, rcv);
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
  }
}

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
  DownCtx c;
#pragma unroll
  for (int k = 0; k < 9; ++k) c.s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  const int T = L.T, M = MG_NET_MARGIN;
#pragma unroll
  for (int k = 0; k < 9; ++k) c.wi[k] = (HK == HK_TABLE && T == MG_PROXY) ? L.W[k * T * T + M * T + M] : 0.f;
  c.omega = omega;
  c.n = n;
  c.R0 = R0;
  c.rc_out = probs[p].lv[l + 1].r;  // per-problem pitched arrays
  c.nc = probs[p].lv[l + 1].n;
  c.pc = probs[p].lv[l + 1].pitch;
  c.pitch = L.pitch;
  c.e_out = L.e;
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
  const int c0 = C0 + SW * w;  // first owned column of the warp
  c.j = c0 - 2 + lane;         // this lane's column
  c.jin = (unsigned)c.j < (unsigned)n;
  c.own = lane >= 2 && lane < 2 + SW && c.jin;
  c.jmargin = T != MG_PROXY || c.j < M || c.j >= n - M;
  c.col = rs + SW * w + 2 + lane;
  // coarse output of the odd lanes 3 .. 27: column c0/2 + (lane - 3)/2
  c.Jc = (c0 >> 1) + ((lane - 3) >> 1);
  c.cown = (lane & 1) && lane >= 3 && lane <= 27 && c.Jc < c.nc;
  // a warp whose points all lie inside the grid (and, for class tables, at least M from
  // its edges) needs neither bounds checks nor table kernels
  const int m = HK == HK_TABLE ? M : 0;
  const bool inner = (HK != HK_TABLE || T == MG_PROXY) && c0 - 2 >= m && c0 + 29 < n - m && R0 - 1 >= m &&
                     R0 + H + 1 < n - m;
  if (inner) sdown_walk<SK, HK, H, G::BW, false>(L, c);
  else sdown_walk<SK, HK, H, G::BW, true>(L, c);
}

// ------------------------------------------------------------------------ k_sup
// Up-sweep of a tiled level (Algorithm 1, correction and post-smoothing): e1 = e + P e_c,
// t = r - A e1, e = e1 + H t on the CTA's rows R0 .. R0+H-1.  Box row q holds grid row
// R0 - 2 + q of e; walking q = 0 .. H+3 the warp forms e1 on box row q, t on q-1 (zero
// outside the grid: H sees the Dirichlet exterior) and the final correction on q-2.  On
// levels >= 1 that correction goes to the level's f array (other CTAs still read e with
// halos); on level 0 (UPDX) it is added to the float-float iterate, read from (xin_hi,
// xin_lo) and written to (xout_hi, xout_lo), the pair of the other cycle parity.
// Prolongation: coarse point I sits at fine 2I+1, so fine row i interpolates coarse rows
// (i-1)>>1 and i>>1: box rows q/2 and q/2+1 of the coarse block for even q, row q/2+1 for
// odd q; hp holds the horizontal interpolation of a coarse row at the lane's column.
struct UpCtx {
  float s[9], wi[9];
  float omega;
  int n, R0, j, pitch;
  bool jin, own, jmargin;
  const float* col;    // e block, this lane's column
  const float* ca;     // coarse block, column (j - 1) >> 1 of row 0
  const float* cb;     // ... column j >> 1
  const float* rin;    // r of this problem (pitched)
  float* fout;         // levels >= 1: final correction
  const float *xin_hi, *xin_lo;
  float *xout_hi, *xout_lo;
};

template <int SK, int HK, int H, int BW, int CBW, bool UPDX, bool EDGE>
__device__ __forceinline__ void sup_walk(const LevelDev& L, const UpCtx& c) {
  Row3 ea, eb;  // e1 on box rows q-2, q-1
  Row3 ta, tb;  // t on box rows q-3, q-2
  ea.l = ea.c = ea.r = 0.f;
  eb = ea;
  ta = ea;
  tb = ea;
  float hP = 0.5f * (c.ca[0] + c.cb[0]);  // coarse box row 0
  // global loads stay unconditional, so the compiler may issue a chunk's loads together:
  // on boundary warps the address is clamped into the grid and the value discarded
  const int jc = EDGE ? min(max(c.j, 0), c.n - 1) : c.j;
#pragma unroll 1
  for (int q0 = 0; q0 < H + 4; q0 += 6) {
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int q = q0 + u;
      if (q < H + 4) {
        float pe;
        if ((u & 1) == 0) {  // q0 is even, so q has the parity of u
          const float hN = 0.5f * (c.ca[(q / 2 + 1) * CBW] + c.cb[(q / 2 + 1) * CBW]);
          pe = 0.5f * (hP + hN);
          hP = hN;
        } else {
          pe = hP;
        }
        const Row3 ec = row3(c.col[q * BW] + pe);  // e1 on box row q (zero outside the grid)
        if (q >= 2) {
          const int it = c.R0 + q - 3;  // t on box row q-1
          const int itc = EDGE ? min(max(it, 0), c.n - 1) : it;
          const float rv = __ldg(c.rin + (size_t)itc * c.pitch + jc);
          float tv = 0.f;
          if (!EDGE || (c.jin && (unsigned)it < (unsigned)c.n)) {
            float a[9];
            stencil_at<SK>(L, c.s, it, c.j, a);
            tv = rv - dot9r(a, ea, eb, ec);
          }
          const Row3 tc = row3(tv);
          if (q >= 4) {
            const int i = c.R0 + q - 4;  // final correction on box row q-2 (the CTA's rows)
            const size_t g = (size_t)(EDGE ? min(i, c.n - 1) : i) * c.pitch + jc;
            float xh = 0.f, xl = 0.f;
            if (UPDX) {
              xh = __ldg(c.xin_hi + g);
              xl = __ldg(c.xin_lo + g);
            }
            if (c.own && (!EDGE || i < c.n)) {
              const bool margin = EDGE && (c.jmargin || i < MG_NET_MARGIN || i >= c.n - MG_NET_MARGIN);
              const float e = ea.c + strip_H<SK, HK>(L, c.s, c.wi, c.omega, i, c.j, margin, ta, tb, tc);
              if (UPDX) {
                float hi = xh, lo = xl, sum, err;
                two_sum(hi, e, sum, err);
                err += lo;
                fast_two_sum(sum, err, hi, lo);
                __stcg(c.xout_hi + g, hi);
                __stcg(c.xout_lo + g, lo);
              } else {
                __stcg(c.fout + g, e);
              }
            }
          }
          ta = tb;
          tb = tc;
        }
        ea = eb;
        eb = ec;
      }
    }
  }
}

template <int SK, int HK, int WPC, int H, bool UPDX>
__global__ void __launch_bounds__(32 * WPC, Strip<WPC, H>::MINB)
    k_sup(const __grid_constant__ CUtensorMap Me, const __grid_constant__ CUtensorMap Mec,
          const ProbDev* __restrict__ probs, ProbState* __restrict__ state, int l, float omega,
          const float* rin_base, const float* xin_hi, const float* xin_lo, float* xout_hi, float* xout_lo,
          const int* __restrict__ act) {
  using G = Strip<WPC, H>;
  constexpr int CBW = G::CW / 2 + 8;  // coarse block: columns C0/2-4 .. C0/2+CW/2+3
  constexpr int CBH = H / 2 + 3;      //               rows    R0/2-2 .. R0/2+H/2
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int ncx = (n + G::CW - 1) / G::CW, ncy = (n + H - 1) / H;
  if ((int)blockIdx.x >= ncx * ncy) return;
  const int R0 = ((int)blockIdx.x / ncx) * H, C0 = ((int)blockIdx.x % ncx) * G::CW;
  __shared__ __align__(128) float es[G::BH * G::BW];
  __shared__ __align__(128) float ecs[CBH * CBW];
  __shared__ __align__(8) uint64_t bar;
  UpCtx c;
#pragma unroll
  for (int k = 0; k < 9; ++k) c.s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  const int T = L.T, M = MG_NET_MARGIN;
#pragma unroll
  for (int k = 0; k < 9; ++k) c.wi[k] = (HK == HK_TABLE && T == MG_PROXY) ? L.W[k * T * T + M * T + M] : 0.f;
  c.omega = omega;
  c.n = n;
  c.R0 = R0;
  c.pitch = L.pitch;
  const size_t po = (size_t)p * n * L.pitch;  // problem offset in the level's batch arrays
  c.rin = UPDX ? rin_base + po : L.r;
  c.fout = L.f;
  if (UPDX) {
    c.xin_hi = xin_hi + po;
    c.xin_lo = xin_lo + po;
    c.xout_hi = xout_hi + po;
    c.xout_lo = xout_lo + po;
  }
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, (G::BH * G::BW + CBH * CBW) * sizeof(float));
    tma_load_3d(es, &Me, &bar, C0 - 4, R0 - 2, p);
    tma_load_3d(ecs, &Mec, &bar, C0 / 2 - 4, R0 / 2 - 2, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c0 = C0 + SW * w;
  c.j = c0 - 2 + lane;
  c.jin = (unsigned)c.j < (unsigned)n;
  c.own = lane >= 2 && lane < 2 + SW && c.jin;
  c.jmargin = T != MG_PROXY || c.j < M || c.j >= n - M;
  c.col = es + SW * w + 2 + lane;
  c.ca = ecs + (SW / 2) * w + ((lane - 3) >> 1) + 4;  // coarse column (j - 1) >> 1
  c.cb = ecs + (SW / 2) * w + ((lane - 2) >> 1) + 4;  // coarse column j >> 1
  // inside the grid: t on rows R0-1 .. R0+H and columns c0-2 .. c0+29; for class tables the
  // smoothed points (the owned ones) at least M from the edges
  bool inner = c0 - 2 >= 0 && c0 + 29 < n && R0 - 1 >= 0 && R0 + H < n;
  if (HK == HK_TABLE) inner = inner && T == MG_PROXY && c0 >= M && c0 + SW <= n - M && R0 >= M && R0 + H <= n - M;
  if (inner) sup_walk<SK, HK, H, G::BW, CBW, UPDX, false>(L, c);
  else sup_walk<SK, HK, H, G::BW, CBW, UPDX, true>(L, c);
}

// ----------------------------------------------------------------------- k_sres
// Residual of the float-float iterate, r = b - A (x_hi + x_lo) (Dot2: exact products and
// sums for x_hi, plain FP32 for the x_lo terms), its norm partial per CTA and, in the last
// CTA of a problem, the stopping test.  A warp owns 30 columns (lane k holds column
// c0 - 1 + k) and walks the rows R0-1 .. R0+H of x; x and b come straight from global
// memory, one coalesced row per load.
// The row walk of k_sres for one lane; EDGE: bounds checks (warps touching the boundary).
// Away from it every lane evaluates its row (lanes 0 and 31 from wrong neighbours) and
// only the owned lanes store and count theirs.
template <int SK, int H, bool EDGE>
__device__ __forceinline__ float sres_walk(const LevelDev& L, const float (&s)[9], const float* xh, const float* xl,
                                           const float* bb, float* rr, int n, int pitch, int R0, int j, bool jin,
                                           bool own) {
  // unconditional loads (clamped into the grid on boundary warps, the value then
  // discarded), so a chunk's loads can be issued together
  const int jc = EDGE ? min(max(j, 0), n - 1) : j;
  auto ld = [&](const float* a, int i) {
    if (!EDGE) return __ldg(a + (size_t)i * pitch + j);
    const float v = __ldg(a + (size_t)min(max(i, 0), n - 1) * pitch + jc);
    return (jin && (unsigned)i < (unsigned)n) ? v : 0.f;
  };
  Row3 ha = row3(ld(xh, R0 - 1)), la = row3(ld(xl, R0 - 1));  // rows i-1 and i of x
  Row3 hb = row3(ld(xh, R0)), lb = row3(ld(xl, R0));
  float acc = 0.f;
#pragma unroll 1
  for (int q0 = 0; q0 < H; q0 += 6) {
#pragma unroll
  for (int u = 0; u < 6; ++u) {
    const int q = q0 + u;
    if (q >= H) break;
    const int i = R0 + q;  // residual on grid row i
    const Row3 hc = row3(ld(xh, i + 1)), lc = row3(ld(xl, i + 1));
    const float bv = ld(bb, i);
    if (!EDGE || (jin && i < n)) {
      float a[9];
      stencil_at<SK>(L, s, i, j, a);
      float hi = bv, lo = 0.f;
      dot2_sub(a[0], ha.l, la.l, hi, lo);
      dot2_sub(a[1], ha.c, la.c, hi, lo);
      dot2_sub(a[2], ha.r, la.r, hi, lo);
      dot2_sub(a[3], hb.l, lb.l, hi, lo);
      dot2_sub(a[4], hb.c, lb.c, hi, lo);
      dot2_sub(a[5], hb.r, lb.r, hi, lo);
      dot2_sub(a[6], hc.l, lc.l, hi, lo);
      dot2_sub(a[7], hc.c, lc.c, hi, lo);
      dot2_sub(a[8], hc.r, lc.r, hi, lo);
      const float r = hi + lo;
      if (own) {
        __stcg(rr + (size_t)i * pitch + j, r);
        acc = fmaf(r, r, acc);
      }
    }
    ha = hb;
    la = lb;
    hb = hc;
    lb = lc;
  }
  }
  return acc;
}

template <int SK, int WPC, int H>
__global__ void __launch_bounds__(32 * WPC, Strip<WPC, H>::MINB)
    k_sres(const ProbDev* __restrict__ probs, ProbState* __restrict__ state, float* __restrict__ partials,
           int ntiles_max, float rtol, int max_cycles, const float* __restrict__ xh_base,
           const float* __restrict__ xl_base, const float* __restrict__ b_base, float* __restrict__ r_base,
           const int* __restrict__ act) {
  constexpr int NT = 32 * WPC, RW = 30, CW = RW * WPC;
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const int n = probs[p].lv[0].n, pitch = probs[p].lv[0].pitch;
  const int ncx = (n + CW - 1) / CW, ncy = (n + H - 1) / H, ntiles = ncx * ncy;
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ncx) * H, C0 = (tile % ncx) * CW;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? probs[p].lv[0].s[k] : 0.f;
  const LevelDev& L = probs[p].lv[0];
  const size_t po = (size_t)p * n * pitch;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c0 = C0 + RW * w;  // first owned column of the warp
  const int j = c0 - 1 + lane;
  const bool jin = (unsigned)j < (unsigned)n;
  const bool own = lane >= 1 && lane < 1 + RW && jin;
  const bool inner = c0 - 1 >= 0 && c0 + 30 < n && R0 - 1 >= 0 && R0 + H < n;
  pdl_wait();
  if (!st_active(state + p)) return;
  const float acc = inner ? sres_walk<SK, H, false>(L, s, xh_base + po, xl_base + po, b_base + po, r_base + po, n,
                                                    pitch, R0, j, jin, own)
                          : sres_walk<SK, H, true>(L, s, xh_base + po, xl_base + po, b_base + po, r_base + po, n,
                                                   pitch, R0, j, jin, own);
  float rhi, rlo;
  if (block_partial_and_last<NT>(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, rhi, rlo)) {
    if (threadIdx.x == 0) decide(state[p], rhi, rlo, rtol, max_cycles);
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

template <int WPC, int H>
static cudaError_t sup_shape(const CycleArgs& a, int l, int parity, dim3 grid) {
  using G = Strip<WPC, H>;
  // the kernel after the cluster tail waits for it by plain stream order (the tail's
  // clusters hold whole SMs; starting early buys nothing there)
  const bool pdl = a.pdl && !(a.ctail && l == a.lstar - 1);
  const CUtensorMap& me = a.maps->se[l];
  const CUtensorMap& mec = a.maps->sec[l];
  const ProbDev* probs = a.probs;
  cudaError_t e = cudaSuccess;
  if (l == 0) {
    const float* rin = parity ? a.r0b : a.r0a;
    const float* xih = parity ? a.xh0b : a.xh0;
    const float* xil = parity ? a.xl0b : a.xl0;
    float* xoh = parity ? a.xh0 : a.xh0b;
    float* xol = parity ? a.xl0 : a.xl0b;
    MG_DISPATCH(a.sk, a.hk,
                (e = launch_pdl(pdl, k_sup<SK_, HK_, WPC, H, true>, grid, dim3(G::NT), 0, a.stream, me, mec, probs,
                                a.state, l, a.omega, rin, xih, xil, xoh, xol, a.active)));
  } else {
    const float* nulc = nullptr;
    float* nul = nullptr;
    MG_DISPATCH(a.sk, a.hk,
                (e = launch_pdl(pdl, k_sup<SK_, HK_, WPC, H, false>, grid, dim3(G::NT), 0, a.stream, me, mec, probs,
                                a.state, l, a.omega, nulc, nulc, nulc, nul, nul, a.active)));
  }
  return e;
}

template <int WPC, int H>
static cudaError_t sres_shape(const CycleArgs& a, const float* xh, const float* xl, float* r, float rtol,
                              int max_cycles, int np) {
  constexpr int CW = 30 * WPC;
  const int n = a.n0;
  const dim3 grid(((n + CW - 1) / CW) * ((n + H - 1) / H), np);
  if (a.sk == SK_CONST)
    return launch_pdl(a.pdl, k_sres<SK_CONST, WPC, H>, grid, dim3(32 * WPC), 0, a.stream, (const ProbDev*)a.probs,
                      a.state, a.partials, a.ntiles_max, rtol, max_cycles, xh, xl, a.b0, r, a.active);
  return launch_pdl(a.pdl, k_sres<SK_FIELD, WPC, H>, grid, dim3(32 * WPC), 0, a.stream, (const ProbDev*)a.probs,
                    a.state, a.partials, a.ntiles_max, rtol, max_cycles, xh, xl, a.b0, r, a.active);
}

void strip_coarse_box(int shape, int* bw, int* bh) {
  int cw, h;
  strip_cta(shape, &cw, &h);
  *bw = cw / 2 + 8;
  *bh = h / 2 + 3;
}

cudaError_t launch_sup(const CycleArgs& a, int l, int parity, int np) {
  int cw, h;
  strip_cta(a.shape, &cw, &h);
  const int n = a.nl[l];
  const dim3 grid(((n + cw - 1) / cw) * ((n + h - 1) / h), np);
  switch (a.shape) {
    case MG_SHAPE_STRIP4x32: return sup_shape<4, 32>(a, l, parity, grid);
    case MG_SHAPE_STRIP8x64: return sup_shape<8, 64>(a, l, parity, grid);
    default: return sup_shape<8, 32>(a, l, parity, grid);
  }
}

cudaError_t launch_sres(const CycleArgs& a, const float* xh, const float* xl, float* r, float rtol, int max_cycles,
                        int np) {
  switch (a.shape) {
    case MG_SHAPE_STRIP4x32: return sres_shape<4, 32>(a, xh, xl, r, rtol, max_cycles, np);
    case MG_SHAPE_STRIP8x64: return sres_shape<8, 64>(a, xh, xl, r, rtol, max_cycles, np);
    default: return sres_shape<8, 32>(a, xh, xl, r, rtol, max_cycles, np);
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
