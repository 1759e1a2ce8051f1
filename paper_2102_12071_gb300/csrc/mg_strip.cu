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
//   k_pdown(l)  the same on constant stencils with a column pair per lane in packed FP32 (60
//               owned columns per warp), each warp walking its rows alone through a ring of
//               8-row copies; bit-identical to the 32 x 32 tiles, the default layout for the
//               launches whose walks are at least 32 rows high
#include <cudaTypedefs.h>

#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_pair.cuh"
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

// ---------------------------------------------------------------------- k_pdown
// The down-sweep of a constant-stencil level in paired warp strips.  Lane k holds the
// column pair (c0 - 2 + 2k, c0 - 1 + 2k), so a warp covers 64 columns, and lanes 1 .. 30
// own the 60 from c0 (the outer lanes carry the halo); every arithmetic step is one packed
// FP32 instruction for both columns, each lane rounded as the scalar instruction, in the
// order of the tile kernels, so e and r_c equal theirs bit for bit.  A warp walks down H
// rows on its own: its rows arrive as 8-row TMA copies (box columns c0-4 .. c0+63) into a
// ring of four stages with one mbarrier each, the copy of a stage going out again as soon
// as the warp has read its last row, and e and r_c leave by coalesced global stores, so no
// CTA-wide barrier is taken.  The launch chooses H so that the walks of all problems fill
// about one wave of resident warps.
constexpr int PS_OWN = 60;               // owned columns per warp
constexpr int PS_BW = 68;                // box columns c0-4 .. c0+63
constexpr int PS_K = 8;                  // rows per copy
constexpr int PS_S = 4;                  // stages per warp
constexpr int PS_WPC = 4;                // warps per CTA
constexpr int PS_MINB = 4;               // resident CTAs per SM the register bound aims at
constexpr int PS_STAGE = PS_K * PS_BW;   // floats per stage
static_assert(PS_STAGE * sizeof(float) % 128 == 0, "stages start 128-byte aligned");
static_assert((PS_BW * sizeof(float)) % 16 == 0 && PS_OWN % 4 == 0, "TMA box and x start 16-byte multiples");

// global stores under a predicate (one predicated instruction each, no branch)
__device__ __forceinline__ void stg2_if(bool p, float* a, float2 v) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.v2.f32 [%1], {%2, %3};\n}" ::"r"((int)p),
               "l"(a), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ void stg_if(bool p, float* a, float v) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.f32 [%1], %2;\n}" ::"r"((int)p), "l"(a),
               "f"(v));
}

// Box row b of the walk holds grid row R0 - 2 + b, and copy c box rows 8c .. 8c+7.  The
// walk keeps r on rows i, i+1 and e on rows i-1, i; the step at box row b (i = R0 - 4 + b)
// reads r on row i+2, forms e = H r on row i+1 (stored on the owned rows), s = r - A e on
// row i and the row sums of the restriction: an even row 2A+2 ends coarse row A (its r_c is
// stored) and starts A+1, an odd row 2A+1 is A's centre row.  Box rows 0 .. 3 start the
// walk; a copy whose eight rows are all steps runs as one unrolled block between the wait
// for it and the sending of its stage's next copy, and the rows before and after such
// copies run one at a time.
template <int HK>
__global__ void __launch_bounds__(32 * PS_WPC, PS_MINB) k_pdown(const __grid_constant__ CUtensorMap Mr,
                                                                const ProbDev* __restrict__ probs,
                                                                ProbState* __restrict__ state, int l, float omega,
                                                                int H, const int* __restrict__ act) {
  __shared__ __align__(128) float rbuf[PS_WPC][PS_S][PS_STAGE];
  __shared__ __align__(8) uint64_t bars[PS_WPC][PS_S];
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int nb = (n + PS_OWN - 1) / PS_OWN, ns = (n + H - 1) / H;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = (int)blockIdx.x * PS_WPC + w;
  if (g >= nb * ns) return;  // the whole warp: nothing below waits for the CTA
  const int R0 = (g / nb) * H, c0 = (g % nb) * PS_OWN;
  const int nc = probs[p].lv[l + 1].n, pc = probs[p].lv[l + 1].pitch;
  float* const rc_out = probs[p].lv[l + 1].r;
  // coarse rows R0/2 .. R0/2 + kend - 1 lie in the coarse grid; the walk reads box rows
  // 0 .. last, which arrive in C copies
  const int kend = min(H / 2, nc - R0 / 2);
  const int last = kend > 0 ? 2 * kend + 4 : 3;
  const int C = last / PS_K + 1;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = L.s[k];
  const int j = c0 - 2 + 2 * lane;  // the lane's columns j, j+1
  const bool inx = (unsigned)j < (unsigned)n, iny = (unsigned)(j + 1) < (unsigned)n;
  // network kernels of the lane's two columns on the rows at least MG_NET_MARGIN from the top
  // and bottom edges (row class MG_NET_MARGIN)
  const int T = L.T, M = MG_NET_MARGIN;
  const int cx = inx ? kclass(j, n, T) : M, cy = iny ? kclass(j + 1, n, T) : M;
  float2 wp[9];
  if (HK == HK_TABLE) {
#pragma unroll
    for (int k = 0; k < 9; ++k) wp[k] = make_float2(L.W[k * T * T + M * T + cx], L.W[k * T * T + M * T + cy]);
  }
  const float2 jw = p2(omega / s[4]);
  float* const buf = rbuf[w][0];
  uint64_t* const bar = bars[w];
  pdl_wait();
  if (!st_active(state + p)) return;
  const bool short_wait = __ldcg(&state[p].short_wait) != 0;
  auto issue = [&](int c) {
    mbar_arrive_expect_tx(&bar[c % PS_S], PS_STAGE * sizeof(float));
    tma_load_3d(buf + (c % PS_S) * PS_STAGE, &Mr, &bar[c % PS_S], c0 - 4, R0 - 2 + c * PS_K, p);
  };
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < PS_S; ++c) mbar_init(&bar[c], 1);
    fence_mbar_init();
    for (int c = 0; c < PS_S && c < C; ++c) issue(c);
  }
  __syncwarp();

  const float* const lrow = buf + 2 + 2 * lane;  // the lane's pair on row 0 of stage 0
  auto at = [&](int b) { return lrow + ((b / PS_K) % PS_S) * PS_STAGE + (b % PS_K) * PS_BW; };
  // a wait that expires clears ok (the walk and further copies stop) and records the copy
  bool ok = true;
  int failed = 0;
  auto wait = [&](int c) {
    if (!ok) return;
    const bool got = !short_wait && mbar_wait(&bar[c % PS_S], (c / PS_S) & 1);
    if (__any_sync(0xffffffffu, !got)) {
      ok = false;
      failed = c;
    }
  };
  auto release = [&](int c) {
    __syncwarp();
    if (ok && lane == 0 && c + PS_S < C) issue(c + PS_S);
  };
  auto load = [&](const float* q) {
    PRow o;
    o.m = ld2(q);
    o.l = q[-1];
    o.r = q[2];
    return o;
  };
  // e = H r on grid row ie from r on rows ie-1 .. ie+1: zero outside the grid; INNER: the
  // row lies at least MG_NET_MARGIN inside the grid
  auto e_row = [&](int ie, bool inner, const PRow& a, const PRow& b, const PRow& c) -> float2 {
    if (HK == HK_JACOBI) return mul2(jw, b.m);  // r is zero outside the grid
    float2 e;
    const int ci = inner ? M : ((unsigned)ie < (unsigned)n ? kclass(ie, n, T) : -1);
    if (ci == M) {
      e = dot9wp(wp, win_rows(a, b, c));
    } else if (ci < 0) {
      e = make_float2(0.f, 0.f);
    } else {
      float2 wr[9];
#pragma unroll
      for (int k = 0; k < 9; ++k)
        wr[k] = make_float2(__ldg(L.W + k * T * T + ci * T + cx), __ldg(L.W + k * T * T + ci * T + cy));
      e = dot9wp(wr, win_rows(a, b, c));
    }
    e.x = inx ? e.x : 0.f;
    e.y = iny ? e.y : 0.f;
    return e;
  };
  auto halo = [&](float2 e) {
    PRow o;
    o.m = e;
    o.l = __shfl_up_sync(0xffffffffu, e.y, 1);
    o.r = __shfl_down_sync(0xffffffffu, e.x, 1);
    return o;
  };
  // e is stored on rows R0 .. e_end-1 by lanes 1 .. 30 as pairs: n is odd and the row pitch
  // a multiple of 32, so a pair that ends at column n writes its zero into the row's padding
  const int e_end = min(R0 + H, n);
  const bool own = lane >= 1 && lane <= 30 && inx;
  float* const e_lane = L.e + (own ? j : 0);
  const size_t epitch = L.pitch;
  const int B = (c0 >> 1) - 1 + lane;  // coarse column of the lane's restriction
  const bool cown = lane >= 1 && lane <= 30 && B < nc;
  float* const rc_lane = rc_out + (cown ? B : 0);

  PRow ra, rb, rc, ea, eb, ec;
  float2 top = make_float2(0.f, 0.f), cen = top;
  // the step at grid row i from box row q, storing e at er (row i+1) and r_c at cr (coarse
  // row i/2 - 1 on even rows); FIRST: i == R0 (no coarse row ends there)
  auto step = [&](const float* q, int i, bool even, bool first, bool inner, float* er, float* cr) {
    rc = load(q);
    const float2 e = e_row(i + 1, inner, ra, rb, rc);
    stg2_if(own && i + 1 < e_end, er, e);
    ec = halo(e);
    const float2 sv = sub2(ra.m, dot9w<false>(s, win_rows(ea, eb, ec)));
    const float z = __shfl_down_sync(0xffffffffu, sv.x, 1);  // s two columns right of the pair
    if (even) {
      const float2 bot = make_float2(sv.x + z, sv.y);
      if (!first) {
        const float edge = (top.y + bot.y) + cen.x;
        const float corner = top.x + bot.x;
        const float v = cen.y + 0.5f * edge + 0.25f * corner;
        stg_if(cown, cr, v);
      }
      top = bot;
    } else {
      cen = make_float2(sv.x + z, sv.y);
    }
    ra = rb;
    rb = rc;
    ea = eb;
    eb = ec;
  };
  // one step with its copy's wait and release
  auto single = [&](int b) {
    const int i = R0 - 4 + b;
    if (b % PS_K == 0) wait(b / PS_K);
    step(at(b), i, (i & 1) == 0, i == R0, false, e_lane + (size_t)(i + 1) * epitch,
         rc_lane + (size_t)((i >> 1) - 1) * pc);
    if (b % PS_K == PS_K - 1) release(b / PS_K);
  };

  wait(0);
  ra = load(at(0));
  rb = load(at(1));
  rc = load(at(2));
  ea = halo(e_row(R0 - 1, false, ra, rb, rc));
  ra = rb;
  rb = rc;
  rc = load(at(3));
  {
    const float2 e = e_row(R0, false, ra, rb, rc);
    stg2_if(own, e_lane + (size_t)R0 * epitch, e);
    eb = halo(e);
  }
  ra = rb;
  rb = rc;
  int b = 4;
  for (; ok && b < PS_K && b <= last; ++b) single(b);
  for (int c = 1; ok && PS_K * c + PS_K - 1 <= last; ++c) {
    wait(c);
    if (!ok) break;
    const float* q = lrow + (c % PS_S) * PS_STAGE;
    const int i0 = R0 - 4 + PS_K * c;  // even
    float* er = e_lane + (size_t)(i0 + 1) * epitch;
    float* cr = rc_lane + (size_t)((i0 >> 1) - 1) * pc;
    if (HK == HK_JACOBI || (i0 + 1 >= M && i0 + PS_K < n - M)) {
#pragma unroll
      for (int t = 0; t < PS_K; ++t) {
        step(q + t * PS_BW, i0 + t, (t & 1) == 0, false, true, er, cr);
        er += epitch;
        if (t & 1) cr += pc;
      }
    } else {
#pragma unroll
      for (int t = 0; t < PS_K; ++t) {
        step(q + t * PS_BW, i0 + t, (t & 1) == 0, false, false, er, cr);
        er += epitch;
        if (t & 1) cr += pc;
      }
    }
    release(c);
    b = PS_K * (c + 1);
  }
  for (; ok && b <= last; ++b) single(b);
  if (!ok) {
    // the wait for copy `failed` expired: mark the problem, then wait for the copies still
    // in flight (those up to failed + PS_S - 1 were sent) before the warp exits
    if (lane == 0) {
      state[p].status = 4;
      state[p].active = 0;
    }
    for (int c = failed; c < failed + PS_S && c < C; ++c) mbar_wait(&bar[c % PS_S], (c / PS_S) & 1);
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

// Rows per warp of a k_pdown launch: the walks of all problems fill about one wave of
// resident warps (at least 8 rows, a multiple of the copy height).
template <int HK>
static int pdown_rows(int n, int np) {
  static int per_sm[64];  // resident CTAs per SM, by device (0 until asked)
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int& b = per_sm[dev & 63];
  if (b == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pdown<HK>, 32 * PS_WPC, 0) != cudaSuccess) b = 1;
  const long long cap = (long long)(nsm > 0 ? nsm : 1) * (b > 0 ? b : 1) * PS_WPC;
  const long long per_seg = (long long)((n + PS_OWN - 1) / PS_OWN) * (np > 0 ? np : 1);
  const long long ns = cap / per_seg > 1 ? cap / per_seg : 1;
  int H = (int)((n + ns - 1) / ns);
  H = (H + PS_K - 1) / PS_K * PS_K;
  return H < PS_K ? PS_K : H;
}

template <int HK>
static cudaError_t pdown_launch(const CycleArgs& a, const CUtensorMap& m, int l, int np) {
  const int n = a.nl[l], H = pdown_rows<HK>(n, np);
  const int warps = ((n + PS_OWN - 1) / PS_OWN) * ((n + H - 1) / H);
  const dim3 grid((warps + PS_WPC - 1) / PS_WPC, np);
  return launch_pdl(a.pdl, k_pdown<HK>, grid, dim3(32 * PS_WPC), 0, a.stream, m, (const ProbDev*)a.probs, a.state, l,
                    a.omega, H, a.active);
}

void strip_box(int shape, int* bw, int* bh) {
  switch (shape) {
    case MG_SHAPE_PSTRIP: *bw = PS_BW; *bh = PS_K; return;
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

// Paired strips pay off when every walk of a one-wave launch is long (a.strip_rows, 32 rows
// by default: four copies); shorter walks (few problems or small levels) spend their time
// starting up, and the 32 x 32 tiles (bit-identical results) take those launches.
bool pdown_applies(const CycleArgs& a, int l, int np) {
  if (a.shape != MG_SHAPE_PSTRIP || a.sk != SK_CONST || (a.hk != HK_JACOBI && a.hk != HK_TABLE)) return false;
  const int H = a.hk == HK_JACOBI ? pdown_rows<HK_JACOBI>(a.nl[l], np) : pdown_rows<HK_TABLE>(a.nl[l], np);
  return H >= a.strip_rows;
}

cudaError_t launch_sdown(const CycleArgs& a, const CUtensorMap& m, int l, int np) {
  if (a.shape == MG_SHAPE_PSTRIP) {
    if (a.sk != SK_CONST) return cudaErrorNotSupported;
    return a.hk == HK_JACOBI ? pdown_launch<HK_JACOBI>(a, m, l, np) : pdown_launch<HK_TABLE>(a, m, l, np);
  }
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
