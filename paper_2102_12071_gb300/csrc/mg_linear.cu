// mg_linear.cu -- the V-cycle with the shared-kernel linear smoother of Sec. 6 (eq.
// full-coarsening-smoother), for sm_103a:
//
//   H v = f_5(f_4(f_3(f_2(f_1(v))))) + f_6(v),  f_k(u)(x) = sum_t phi_k[t] u(x + d_t),
//
// six 3x3 kernels per level shared by every point (and by every problem of a context, or
// one group per problem with net_per_problem), each layer's input zero outside the grid.
// On the levels of side > MG_TAIL_N every smoothing is one tiled kernel (k_lin_Htile): a
// TMA copy brings the input tile with the chain's five-point halo into shared memory, the
// five layers run there on shrinking regions (register windows, three shared loads per
// point), and only H v leaves the SM -- 8 bytes per point instead of 8 per layer.  The
// residual-and-restriction, prolongation, update and compensated residual are point
// kernels on a 2-D grid (32 x 8 threads per CTA, problem in blockIdx.z).  The levels below
// run in the one-CTA tail (mg_tail.cuh), which holds the chain in shared memory.  The
// level-0 update and the compensated residual with the stopping test follow the same
// conventions as the tiled path (iterate and residual alternate between two arrays by
// cycle parity).
#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_ops.cuh"
#include "mg_pair.cuh"
#include "mg_reduce.cuh"
#include "mg_tile.cuh"
#include "mg_tma.cuh"

namespace mg {

constexpr int LT = 256;  // threads per CTA of the point kernels
constexpr int PX = 32, PY = 8, RY = 4;  // point kernels: 32 x 8 threads, 4 rows each (32 x 32 points)

// problem of this CTA (-1: none); the launch index is blockIdx.y or blockIdx.z
__device__ __forceinline__ int lin_problem(const ProbState* state, const int* act, int pfix, int idx) {
  if (pfix >= 0) return pfix;
  const int p = act ? act[idx] : idx;
  return st_active(state + p) ? p : -1;
}

__device__ __forceinline__ float tap_at(const float* v, int pitch, int n, int i, int j) {
  return ((unsigned)i < (unsigned)n && (unsigned)j < (unsigned)n) ? v[(size_t)i * pitch + j] : 0.f;
}

// sum_t w[t] v(i + di_t, j + dj_t), centre tap first (the order of every other stencil sum)
__device__ __forceinline__ float conv_at(const float (&w)[9], const float* v, int pitch, int n, int i, int j) {
  float acc = w[4] * v[(size_t)i * pitch + j];
  acc = fmaf(w[0], tap_at(v, pitch, n, i - 1, j - 1), acc);
  acc = fmaf(w[1], tap_at(v, pitch, n, i - 1, j), acc);
  acc = fmaf(w[2], tap_at(v, pitch, n, i - 1, j + 1), acc);
  acc = fmaf(w[3], tap_at(v, pitch, n, i, j - 1), acc);
  acc = fmaf(w[5], tap_at(v, pitch, n, i, j + 1), acc);
  acc = fmaf(w[6], tap_at(v, pitch, n, i + 1, j - 1), acc);
  acc = fmaf(w[7], tap_at(v, pitch, n, i + 1, j), acc);
  acc = fmaf(w[8], tap_at(v, pitch, n, i + 1, j + 1), acc);
  return acc;
}

// A v at (i, j): constant taps s, or the point's taps of the stencil field
template <int SK>
__device__ __forceinline__ float apply_A_at(const LevelDev& L, const float (&s)[9], const float* v, int pitch, int i,
                                            int j) {
  const int n = L.n;
  float a[9];
  if (SK == SK_CONST) {
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = s[k];
  } else {
    const size_t nn = (size_t)n * n, q = (size_t)i * n + j;
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = __ldg(L.st + k * nn + q);
  }
  return conv_at(a, v, pitch, n, i, j);
}

// ------------------------------------------------------------------ chain passes
// MODE 0: dst = f_k(src); 1: dst = f_5(src) + f_6(src2); 2: dst += f_5(src) + f_6(src2),
// with the weights of level l of the CTA's problem.  With pfix >= 0 the arrays are problem
// pfix's dense n x n vectors (pitch = n).
template <int MODE>
__global__ void __launch_bounds__(LT) k_lin_conv(const ProbDev* __restrict__ probs, int l, int k, int n, int pitch,
                                                 const ProbState* __restrict__ state, const int* __restrict__ act,
                                                 int pfix, const float* src, const float* src2, float* dst) {
  pdl_trigger();
  const int q = blockIdx.x * LT + threadIdx.x;
  // the weights never change after setup, so they load before the wait
  const int pw = pfix >= 0 ? pfix : (act ? act[blockIdx.y] : blockIdx.y);
  const float* phi = probs[pw].lv[l].W;
  float w[9], w6[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    w[t] = phi[9 * k + t];
    w6[t] = MODE ? phi[45 + t] : 0.f;
  }
  pdl_wait();
  const int p = lin_problem(state, act, pfix, blockIdx.y);
  if (p < 0 || q >= n * n) return;
  const size_t off = pfix >= 0 ? 0 : (size_t)p * n * pitch;
  const int i = q / n, j = q % n;
  const size_t o = off + (size_t)i * pitch + j;
  float h = conv_at(w, src + off, pitch, n, i, j);
  if (MODE) h += conv_at(w6, src2 + off, pitch, n, i, j);
  dst[o] = MODE == 2 ? dst[o] + h : h;
}

// r_{l+1} = P^T (r - A e), a thread per coarse point of RY rows: the residual on the 3 x 3
// fine points of its restriction stencil (fine 2I+1+d, all inside the grid) from e's 5 x 5
// neighbourhood, then the restriction of Sec. 6.1 in the tile kernels' summation order.
template <int SK>
__global__ void __launch_bounds__(LT) k_lin_restrict(const ProbDev* __restrict__ probs,
                                                     const ProbState* __restrict__ state, const int* __restrict__ act,
                                                     int l, const float* r, const float* e, float* rc) {
  pdl_trigger();
  pdl_wait();
  const int p = lin_problem(state, act, -1, blockIdx.z);
  if (p < 0) return;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, pitch = L.pitch, nc = probs[p].lv[l + 1].n, pc = probs[p].lv[l + 1].pitch;
  const int J = blockIdx.x * PX + threadIdx.x;
  if (J >= nc) return;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  const size_t off = (size_t)p * n * pitch;
  const float* rp = r + off;
  const float* ep = e + off;
  for (int y = 0; y < RY; ++y) {
    const int I = blockIdx.y * PY * RY + y * PY + threadIdx.y;
    if (I >= nc) break;
    float sv[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int fi = 2 * I + a, fj = 2 * J + b;
        sv[3 * a + b] = rp[(size_t)fi * pitch + fj] - apply_A_at<SK>(L, s, ep, pitch, fi, fj);
      }
    rc[(size_t)p * nc * pc + (size_t)I * pc + J] = restrict_at(sv + 4, 3);
  }
}

// e_l += P e_{l+1} (bilinear, Sec. 6.1), a thread per fine point of RY rows, coarse values
// zero outside the coarse grid; the arithmetic of prolong_at
__global__ void __launch_bounds__(LT) k_lin_prolong(const ProbDev* __restrict__ probs,
                                                    const ProbState* __restrict__ state, const int* __restrict__ act,
                                                    int l, float* e, const float* ec) {
  pdl_trigger();
  pdl_wait();
  const int p = lin_problem(state, act, -1, blockIdx.z);
  if (p < 0) return;
  const int n = probs[p].lv[l].n, pitch = probs[p].lv[l].pitch;
  const int nc = probs[p].lv[l + 1].n, pc = probs[p].lv[l + 1].pitch;
  const int j = blockIdx.x * PX + threadIdx.x;
  if (j >= n) return;
  const float* c = ec + (size_t)p * nc * pc;
  float* ep = e + (size_t)p * n * pitch;
  const int Ja = (j - 1) >> 1;
  for (int y = 0; y < RY; ++y) {
    const int i = blockIdx.y * PY * RY + y * PY + threadIdx.y;
    if (i >= n) break;
    const int Ia = (i - 1) >> 1;
    const float b00 = tap_at(c, pc, nc, Ia, Ja), b01 = tap_at(c, pc, nc, Ia, Ja + 1);
    const float b10 = tap_at(c, pc, nc, Ia + 1, Ja), b11 = tap_at(c, pc, nc, Ia + 1, Ja + 1);
    float v;
    if (i & 1) v = (j & 1) ? b00 : 0.5f * (b00 + b01);
    else v = (j & 1) ? 0.5f * (b00 + b10) : 0.25f * ((b00 + b01) + (b10 + b11));
    ep[(size_t)i * pitch + j] += v;
  }
}

// t = r - A e on one level, a thread per point of RY rows
template <int SK>
__global__ void __launch_bounds__(LT) k_lin_residual(const ProbDev* __restrict__ probs,
                                                     const ProbState* __restrict__ state, const int* __restrict__ act,
                                                     int l, const float* r, const float* e, float* t) {
  pdl_trigger();
  pdl_wait();
  const int p = lin_problem(state, act, -1, blockIdx.z);
  if (p < 0) return;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, pitch = L.pitch;
  const int j = blockIdx.x * PX + threadIdx.x;
  if (j >= n) return;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  const size_t off = (size_t)p * n * pitch;
  for (int y = 0; y < RY; ++y) {
    const int i = blockIdx.y * PY * RY + y * PY + threadIdx.y;
    if (i >= n) break;
    const size_t o = off + (size_t)i * pitch + j;
    t[o] = r[o] - apply_A_at<SK>(L, s, e + off, pitch, i, j);
  }
}

// dst (=, or += with ACC) (omega / D) u: weighted Jacobi (Sec. 2.1) on the batched level
// path (smoothing with nu1, nu2 > 1), the arithmetic of the tiled kernels' Jacobi step
template <int SK, bool ACC>
__global__ void __launch_bounds__(LT) k_jac_H(const ProbDev* __restrict__ probs, const ProbState* __restrict__ state,
                                              const int* __restrict__ act, int l, float omega, const float* u,
                                              float* dst) {
  pdl_trigger();
  pdl_wait();
  const int p = lin_problem(state, act, -1, blockIdx.z);
  if (p < 0) return;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, pitch = L.pitch;
  const int j = blockIdx.x * PX + threadIdx.x;
  if (j >= n) return;
  const size_t off = (size_t)p * n * pitch, nn = (size_t)n * n;
  for (int y = 0; y < RY; ++y) {
    const int i = blockIdx.y * PY * RY + y * PY + threadIdx.y;
    if (i >= n) break;
    const float d = (SK == SK_CONST) ? L.s[4] : __ldg(L.st + 4 * nn + (size_t)i * n + j);
    const size_t o = off + (size_t)i * pitch + j;
    const float h = (omega / d) * u[o];
    dst[o] = ACC ? dst[o] + h : h;
  }
}

// dst = K_k(src) (MODE 0) or dst += K_k(src) (MODE 2): one layer of the three-kernel stack
// (MG_NET_CONV3), the kernel of point x is W[9k .. 9k+8](x) of the level's [27][n][n] field,
// src zero outside the grid
template <int MODE>
__global__ void __launch_bounds__(LT) k_stack_conv(const ProbDev* __restrict__ probs,
                                                   const ProbState* __restrict__ state, const int* __restrict__ act,
                                                   int l, int k, const float* src, float* dst) {
  pdl_trigger();
  pdl_wait();
  const int p = lin_problem(state, act, -1, blockIdx.z);
  if (p < 0) return;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, pitch = L.pitch;
  const int j = blockIdx.x * PX + threadIdx.x;
  if (j >= n) return;
  const size_t off = (size_t)p * n * pitch, nn = (size_t)n * n;
  const float* Wk = L.W + (size_t)9 * k * nn;
  for (int y = 0; y < RY; ++y) {
    const int i = blockIdx.y * PY * RY + y * PY + threadIdx.y;
    if (i >= n) break;
    float w[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) w[t] = __ldg(Wk + t * nn + (size_t)i * n + j);
    const float h = conv_at(w, src + off, pitch, n, i, j);
    float* d = dst + off + (size_t)i * pitch + j;
    *d = MODE == 2 ? *d + h : h;
  }
}

// ------------------------------------------------------------------ the tiled chain
// One CTA per 32 x 32 output tile.  Coordinates below are in the frame of the input tile
// u: row 0 = grid row R0 - 5, column 0 = grid column C0 - 8 (the TMA box starts 8 columns
// left so that its x is 16-byte aligned).  Layer k (k = 1..4) covers the tile grown by
// 5 - k points; the output covers rows [5, 37), columns [8, 40).
constexpr int HT = 32, HH = 5, HR = HT + 2 * HH;  // tile, halo, rows of u
constexpr int HXU = 56;                            // u: row stride of the TMA box

__device__ __forceinline__ bool lin_inside(int i, int j, int n) {
  return (unsigned)i < (unsigned)n && (unsigned)j < (unsigned)n;
}

// The tiled chain runs with two adjacent columns per thread in packed FP32 (mg_pair.cuh),
// 128 threads per tile.  Layer L (L = 1..4) covers frame rows [L, 42 - L) and columns
// [L + 3, 45 - L) in pairs (c, c+1), c = L + 3 + 2q, and writes a buffer whose origin is
// (L, L + 3): the pair's own store is an aligned 64-bit access, and so are the next
// layer's window rows (its column c - 1 is even there).  Layer 1 reads u, whose frame is
// the TMA box: its windows (and f6's) are one 64-bit and two 32-bit loads.  Layers 1 and
// 3 write one buffer, 2 and 4 the other.
constexpr int LTP = 128;  // threads per CTA of the tiled chain kernels
constexpr int BX = 40;    // row stride of the layer buffers

template <int L, int K, bool MASK>
__device__ __forceinline__ void lin_layer2(const float* in, float* out, const float* wsm, int R0, int C0, int n) {
  constexpr int S = HR - 2 * L, NQ = S / 2, NS = (S + K - 1) / K;
  constexpr int XI = L == 1 ? HXU : BX, RI = L == 1 ? 0 : L - 1, CI = L == 1 ? 0 : L + 2;
  static_assert(16 * NS + (NQ - 16) * NS <= LTP, "layer needs more threads than the CTA has");
  int q, strip;
  if (!chunk_item<NQ, NS>(threadIdx.x, q, strip)) return;
  float w[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = wsm[k];
  const int r0 = L + strip * K, c = L + 3 + 2 * q;
  const float* src = in + (r0 - 1 - RI) * XI + (L == 1 ? c : c - 1 - CI);  // window row a
  float* dst = out + (r0 - L) * BX + 2 * q;
  Win2 v;
  if (L == 1) {
    row_even(src, v.la, v.ma, v.ra);
    row_even(src + XI, v.lb, v.mb, v.rb);
  } else {
    row_odd(src, v.la, v.ma, v.ra);
    row_odd(src + XI, v.lb, v.mb, v.rb);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (S % K == 0 || strip * K + k < S) {
      if (L == 1) row_even(src + (k + 2) * XI, v.lc, v.mc, v.rc);
      else row_odd(src + (k + 2) * XI, v.lc, v.mc, v.rc);
      float2 val = dot9w<L != 1>(w, v);
      if (MASK) {
        const int i = R0 - HH + r0 + k, j = C0 - 8 + c;
        if (!lin_inside(i, j, n)) val.x = 0.f;
        if (!lin_inside(i, j + 1, n)) val.y = 0.f;
      }
      st2(dst + k * BX, val);
      v.shift();
    }
  }
}

// dst (=, or += with ACC, or base + with base: four rows per thread) f_5(w_4) + f_6(u) on
// the tile's points inside the grid, pair q = grid columns C0 + 2q, C0 + 2q + 1: one window
// and one kernel live at a time (f_5 over layer 4's buffer first, then f_6 over u)
template <bool MASK, bool ACC>
__device__ __forceinline__ void lin_out2(const float* w4, const float* u, const float* ph, int R0, int C0, int n,
                                         float* dst, int pitch, const float2* base) {
  constexpr int K = 4;
  const int q = threadIdx.x & 15, t0 = (threadIdx.x >> 4) * K, r = HH + t0, c = 8 + 2 * q;
  float2 h[K];
  float w[9];
  Win2 v;
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = ph[36 + k];
  const float* a = w4 + (r - 1 - 4) * BX + 2 * q;  // layer 4's origin (4, 7): column c-1 is 2q
  row_odd(a, v.la, v.ma, v.ra);
  row_odd(a + BX, v.lb, v.mb, v.rb);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    row_odd(a + (k + 2) * BX, v.lc, v.mc, v.rc);
    h[k] = dot9w<true>(w, v);
    v.shift();
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = ph[45 + k];
  const float* b = u + (r - 1) * HXU + c;
  row_even(b, v.la, v.ma, v.ra);
  row_even(b + HXU, v.lb, v.mb, v.rb);
  const int j = C0 + 2 * q;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    row_even(b + (k + 2) * HXU, v.lc, v.mc, v.rc);
    const int i = R0 + t0 + k;
    const float2 hv = add2(h[k], dot9w<false>(w, v));
    float* d = dst + (size_t)i * pitch + j;
    if (!MASK) {
      st2(d, base ? add2(base[k], hv) : (ACC ? add2(ld2(d), hv) : hv));
    } else {
      if (lin_inside(i, j, n)) d[0] = base ? base[k].x + hv.x : (ACC ? d[0] + hv.x : hv.x);
      if (lin_inside(i, j + 1, n)) d[1] = base ? base[k].y + hv.y : (ACC ? d[1] + hv.y : hv.y);
    }
    v.shift();
  }
}

template <bool MASK, bool ACC>
__device__ __forceinline__ void lin_chain(const float* U, float* BA, float* BB, const float* ph, int R0, int C0, int n,
                                          float* dst, int pitch, const float2* base = nullptr) {
  lin_layer2<1, 7, MASK>(U, BA, ph, R0, C0, n);
  __syncthreads();
  lin_layer2<2, 7, MASK>(BA, BB, ph + 9, R0, C0, n);
  __syncthreads();
  lin_layer2<3, 6, MASK>(BB, BA, ph + 18, R0, C0, n);
  __syncthreads();
  lin_layer2<4, 5, MASK>(BA, BB, ph + 27, R0, C0, n);
  __syncthreads();
  lin_out2<MASK, ACC>(BB, U, ph, R0, C0, n, dst, pitch, base);
}

// ------------------------------------------------------------- the fused up-sweep
// Post-smoothing of a level in one kernel (the linear smoother's counterpart of k_up):
// e1 = e + P e_c on the tile and a six-point halo, t = r - A e1 on the chain's input region
// (zero outside the grid), then e1 + H t on the tile, written to an array of its own (other
// CTAs still read e with halos).  Frames: e1 rows from R0 - 6, columns from C0 - 8 (stride
// 48, 44 rows); t in the chain's input frame (rows from R0 - 5, stride 56), computed in
// place over the TMA copy of r; the coarse tile from (R0/2 - 4, C0/2 - 4), 24 x 24.
constexpr int UE_H = HR + 2, UE_X = 48, UC = 24;

template <int SK, bool MASK>
__device__ __forceinline__ void up_prepare(const LevelDev& L, const float (&s)[9], float* E1, float* U,
                                           const float* ecs, int R0, int C0, int n) {
  // e1 = e + P e_c on rows R0-6 .. R0+37, columns C0-6 .. C0+37 (e and e_c are zero outside
  // their grids, so is P e_c outside the fine grid).  Pair q is e1's columns 2 + 2q (an even
  // grid column) and 3 + 2q, whose bilinear weights read coarse box columns (q, q+1) and
  // (q+1, q+1); strips of 10 rows from even offsets read coarse box rows 5 s .. 5 s + 5 (row
  // 2m reads coarse rows m, m+1; row 2m+1 coarse row m+1 twice), and the sum of a coarse row's
  // pair serves two fine rows.  P e_c = ((c_aa + c_ab) + (c_ba + c_bb)) / 4 with coincident
  // indices repeated, which equals the one-, two- and four-point forms exactly.
  {
    constexpr int NQ = 22, KS = 10, NS = (UE_H + KS - 1) / KS;
    static_assert(NQ * NS <= LTP, "prolongation needs more threads than the CTA has");
    if ((int)threadIdx.x < NQ * NS) {
      const int q = threadIdx.x % NQ, s5 = threadIdx.x / NQ;
      const float* cb = ecs + 5 * s5 * UC + q;
      float* ep = E1 + KS * s5 * UE_X + 2 + 2 * q;
      float2 S[KS / 2 + 1];
#pragma unroll
      for (int m = 0; m <= KS / 2; ++m) {
        if (5 * s5 + m < UC) {
          const float a = cb[m * UC], b = cb[m * UC + 1];
          S[m] = add2(make_float2(a, b), p2(b));
        }
      }
#pragma unroll
      for (int k = 0; k < KS; ++k)
        if (KS * s5 + k < UE_H)
          st2(ep + k * UE_X, fma2(p2(0.25f), add2(S[(k + 1) >> 1], S[(k >> 1) + 1]), ld2(ep + k * UE_X)));
    }
  }
  __syncthreads();
  // t = r - A e1 on the chain's input region (frame rows 0..41, columns 3..44) in pairs
  // (3 + 2q, 4 + 2q), K rows per thread with a register window over e1 (e1's row = t's
  // row + 1; column c - 1 is even there)
  constexpr int S = HR, NQ = S / 2, K = 7, NS = (S + K - 1) / K;
  static_assert(16 * NS + (NQ - 16) * NS <= LTP, "residual needs more threads than the CTA has");
  int q, strip;
  if (chunk_item<NQ, NS>(threadIdx.x, q, strip)) {
    const int t0 = strip * K, c = 3 + 2 * q;
    const float* src = E1 + t0 * UE_X + c - 1;
    Win2 v;
    row_odd(src, v.la, v.ma, v.ra);
    row_odd(src + UE_X, v.lb, v.mb, v.rb);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (t0 + k < S) {
        row_odd(src + (k + 2) * UE_X, v.lc, v.mc, v.rc);
        const int i = R0 - HH + t0 + k, j = C0 - 8 + c;
        float* tp = U + (t0 + k) * HXU + c;
        float2 av;
        if (SK == SK_CONST) {
          av = dot9w<true>(s, v);
        } else {
          const size_t nn = (size_t)n * n;
          float a0[9], a1[9];
          const bool in0 = !MASK || lin_inside(i, j, n), in1 = !MASK || lin_inside(i, j + 1, n);
#pragma unroll
          for (int z = 0; z < 9; ++z) {
            a0[z] = in0 ? __ldg(L.st + z * nn + (size_t)i * n + j) : 0.f;
            a1[z] = in1 ? __ldg(L.st + z * nn + (size_t)i * n + j + 1) : 0.f;
          }
          av = make_float2(dot9(a0, lane_win(v, 0)), dot9(a1, lane_win(v, 1)));
        }
        float2 tv = sub2(make_float2(tp[0], tp[1]), av);
        if (MASK) {
          if (!lin_inside(i, j, n)) tv.x = 0.f;
          if (!lin_inside(i, j + 1, n)) tv.y = 0.f;
        }
        tp[0] = tv.x;
        tp[1] = tv.y;
        v.shift();
      }
    }
  }
  __syncthreads();
}

// out = e1 + H t on level l (fused prolongation, residual and post-smoothing);
// mE: e_l with the six-point halo, mR: r_l (the chain's input box), mC: the coarse tile
template <int SK>
__global__ void __launch_bounds__(LTP, 6) k_lin_Uptile(const __grid_constant__ CUtensorMap mE,
                                                       const __grid_constant__ CUtensorMap mR,
                                                       const __grid_constant__ CUtensorMap mC,
                                                       const ProbDev* __restrict__ probs, ProbState* __restrict__ state,
                                                       const int* __restrict__ act, int l, float* __restrict__ out) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, pitch = L.pitch, ntx = (n + HT - 1) / HT;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * HT, C0 = (tile % ntx) * HT;
  __shared__ __align__(128) float U[HR * HXU];
  __shared__ __align__(128) float E1[UE_H * UE_X];
  __shared__ __align__(128) float ecs[UC * UC];
  __shared__ __align__(16) float BA[(HR - 2) * BX];
  __shared__ __align__(16) float BB[(HR - 4) * BX];
  __shared__ float ph[MG_NPARAMS_LIN];
  __shared__ __align__(8) uint64_t bar;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  if (threadIdx.x < MG_NPARAMS_LIN) ph[threadIdx.x] = L.W[threadIdx.x];  // weights never change
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, (HR * HXU + UE_H * UE_X + UC * UC) * sizeof(float));
    tma_load_3d(U, &mR, &bar, C0 - 8, R0 - HH, p);
    tma_load_3d(E1, &mE, &bar, C0 - 8, R0 - HH - 1, p);
    tma_load_3d(ecs, &mC, &bar, C0 / 2 - 4, R0 / 2 - 4, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  const bool inner = R0 >= HH + 1 && C0 >= HH + 1 && R0 + HT + HH + 1 <= n && C0 + HT + HH + 1 <= n;
  if (inner) up_prepare<SK, false>(L, s, E1, U, ecs, R0, C0, n);
  else up_prepare<SK, true>(L, s, E1, U, ecs, R0, C0, n);
  // e1 on the output points of this thread (lin_out2's mapping), then the chain on t
  float2 e1c[4];
  {
    const int q = threadIdx.x & 15, t0 = (threadIdx.x >> 4) * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) e1c[k] = ld2(E1 + (t0 + k + HH + 1) * UE_X + 8 + 2 * q);
  }
  float* d = out + (size_t)p * n * pitch;
  if (inner) lin_chain<false, false>(U, BA, BB, ph, R0, C0, n, d, pitch, e1c);
  else lin_chain<true, false>(U, BA, BB, ph, R0, C0, n, d, pitch, e1c);
}

// dst (=, or += with ACC) H u on level l; mu: the tensor map of u's level array
template <bool ACC>
__global__ void __launch_bounds__(LTP, 8) k_lin_Htile(const __grid_constant__ CUtensorMap mu,
                                                      const ProbDev* __restrict__ probs, ProbState* __restrict__ state,
                                                      const int* __restrict__ act, int l, float* __restrict__ dst) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, pitch = L.pitch, ntx = (n + HT - 1) / HT;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * HT, C0 = (tile % ntx) * HT;
  __shared__ __align__(128) float U[HR * HXU];
  __shared__ __align__(16) float BA[(HR - 2) * BX];
  __shared__ __align__(16) float BB[(HR - 4) * BX];
  __shared__ float ph[MG_NPARAMS_LIN];
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x < MG_NPARAMS_LIN) ph[threadIdx.x] = L.W[threadIdx.x];  // weights never change
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, HR * HXU * sizeof(float));
    tma_load_3d(U, &mu, &bar, C0 - 8, R0 - HH, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  float* d = dst + (size_t)p * n * pitch;
  if (R0 >= HH && C0 >= HH && R0 + HT + HH <= n && C0 + HT + HH <= n)
    lin_chain<false, ACC>(U, BA, BB, ph, R0, C0, n, d, pitch);
  else
    lin_chain<true, ACC>(U, BA, BB, ph, R0, C0, n, d, pitch);
}

// ------------------------------------------------------------- tiled restriction
// r_{l+1} = P^T (r - A e) after the pre-smoothing, on constant stencils: one 32 x 32 fine
// tile (16 x 16 coarse points) per CTA of 128 threads.  TMA copies of r (rows R0 .. R0+32)
// and e (rows R0-1 .. R0+33), both over columns C0-4 .. C0+35; s = r - A e on rows R0 ..
// R0+32 and box columns 4 .. 37 in pairs (4 + 2q, 5 + 2q) over r in place (the pair's own
// values are aligned 64-bit accesses, its window rows one 64-bit and two single loads); the
// restriction two coarse points per thread (the order of restrict_at); r_c out by a TMA
// store.  Every coarse point inside the grid reads fine points inside it only, and the store
// drops coarse points outside, so no masking is needed.
constexpr int RW = 40, RRH = HT + 1, REH = HT + 3, RCT = HT / 2;

__global__ void __launch_bounds__(LTP, 8) k_lin_restrict_tile(const __grid_constant__ CUtensorMap mR,
                                                              const __grid_constant__ CUtensorMap mE,
                                                              const __grid_constant__ CUtensorMap mRc,
                                                              const ProbDev* __restrict__ probs,
                                                              ProbState* __restrict__ state,
                                                              const int* __restrict__ act, int l) {
  pdl_trigger();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, ntx = (n + HT - 1) / HT;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * HT, C0 = (tile % ntx) * HT;
  __shared__ __align__(128) float rs[RRH * RW];
  __shared__ __align__(128) float es[REH * RW];
  __shared__ __align__(128) float rco[RCT * RCT];
  __shared__ __align__(8) uint64_t bar;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = L.s[k];
  pdl_wait();
  if (!st_active(state + p)) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, (RRH + REH) * RW * sizeof(float));
    tma_load_3d(rs, &mR, &bar, C0 - 4, R0, p);
    tma_load_3d(es, &mE, &bar, C0 - 4, R0 - 1, p);
  }
  __syncthreads();
  if (!tile_wait(&bar, state[p])) return;
  {
    constexpr int NQ = 17, K = 5, NS = (RRH + K - 1) / K;
    static_assert(16 * NS + (NQ - 16) * NS <= LTP, "residual needs more threads than the CTA has");
    int q, strip;
    if (chunk_item<NQ, NS>(threadIdx.x, q, strip)) {
      const int t0 = strip * K, c = 4 + 2 * q;
      const float* w = es + t0 * RW + c;  // window row a of s row t0 (e's row 0 is R0 - 1)
      float* rp = rs + t0 * RW + c;
      Win2 v;
      row_even(w, v.la, v.ma, v.ra);
      row_even(w + RW, v.lb, v.mb, v.rb);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (t0 + k < RRH) {
          row_even(w + (k + 2) * RW, v.lc, v.mc, v.rc);
          st2(rp + k * RW, sub2(ld2(rp + k * RW), dot9w<false>(s, v)));
          v.shift();
        }
      }
    }
  }
  __syncthreads();
  {
    // coarse column b = lane of a half-warp, coarse rows a and a + 8: fine rows 2a .. 2a+2
    // and columns 2b .. 2b+2 of the tile (one 64-bit and one single load per row), the order
    // of restrict_at
    const int bq = threadIdx.x & 15, a0 = threadIdx.x >> 4;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = a0 + 8 * h;
      const float* c = rs + 2 * a * RW + 2 * bq + 4;
      float2 u[3];
      float z[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        u[q] = ld2(c + q * RW);
        z[q] = c[q * RW + 2];
      }
      const float edge = (u[0].y + u[2].y) + (u[1].x + z[1]);
      const float corner = (u[0].x + z[0]) + (u[2].x + z[2]);
      rco[a * RCT + bq] = u[1].y + 0.5f * edge + 0.25f * corner;
    }
  }
  fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    tma_store_3d(&mRc, rco, C0 / 2, R0 / 2, p);
    tma_store_commit();
    tma_store_wait();
  }
}

// phi[l] <- the parameters of H^T: (f_5 .. f_1 f_6 reversed)^T = f_1^T .. f_5^T + f_6^T,
// and f^T is the correlation with the mirrored kernel (tap 8 - t)
__global__ void k_lin_transpose(float* phi, int nlev) {
  const int l = blockIdx.x;
  if (l >= nlev || threadIdx.x != 0) return;
  float* p = phi + (size_t)l * MG_NPARAMS_LIN;
  float tmp[MG_NPARAMS_LIN];
  for (int k = 0; k < 5; ++k)
    for (int t = 0; t < 9; ++t) tmp[9 * k + t] = p[9 * (4 - k) + 8 - t];
  for (int t = 0; t < 9; ++t) tmp[45 + t] = p[45 + 8 - t];
  for (int q = 0; q < MG_NPARAMS_LIN; ++q) p[q] = tmp[q];
}

// ---------------------------------------------------------------- launchers
static inline int nlaunch(const CycleArgs& a) { return (a.active && a.nactive > 0) ? a.nactive : a.nprob; }

static dim3 point_grid(int n, int np) { return dim3((n + PX - 1) / PX, (n + PY * RY - 1) / (PY * RY), np); }

// dst (=, or += with acc) H u on level l over the launch set: one tiled kernel
static cudaError_t lin_H(const CycleArgs& a, int l, const CUtensorMap& mu, float* dst, bool acc, int cls) {
  const int nt = (a.nl[l] + HT - 1) / HT;
  const dim3 grid(nt * nt, nlaunch(a));
  a.prof->launches++;
  a.prof->begin(cls, a.stream);
  const cudaError_t e =
      acc ? launch_pdl(a.pdl, k_lin_Htile<true>, grid, dim3(LTP), 0, a.stream, mu, (const ProbDev*)a.probs, a.state,
                       a.active, l, dst)
          : launch_pdl(a.pdl, k_lin_Htile<false>, grid, dim3(LTP), 0, a.stream, mu, (const ProbDev*)a.probs, a.state,
                       a.active, l, dst);
  a.prof->end(a.stream);
  return e;
}

// dst (=, or += with acc) H u on level l: the tiled chain (linear smoother, u one of the
// arrays of a tensor map in LinMaps) or weighted Jacobi
static cudaError_t smooth_H(const CycleArgs& a, int l, const float* u, const CUtensorMap& mu, float* dst, bool acc,
                            int cls) {
  if (a.hk == HK_LINEAR) return lin_H(a, l, mu, dst, acc, cls);
  if (a.hk == HK_STACK3) {  // K3(K2(K1 u)) through the scratch vectors
    const dim3 grid = point_grid(a.nl[l], nlaunch(a));
    const ProbDev* probs = a.probs;
    const ProbState* cst = a.state;
    const float* src = u;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      float* out = k == 2 ? dst : (k == 0 ? a.lin_wa : a.lin_wb);
      a.prof->launches++;
      a.prof->begin(cls, a.stream);
      if (k < 2)
        e = launch_pdl(a.pdl, k_stack_conv<0>, grid, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l, k, src, out);
      else if (acc)
        e = launch_pdl(a.pdl, k_stack_conv<2>, grid, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l, k, src, out);
      else
        e = launch_pdl(a.pdl, k_stack_conv<0>, grid, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l, k, src, out);
      a.prof->end(a.stream);
      src = out;
    }
    return e;
  }
  a.prof->launches++;
  a.prof->begin(cls, a.stream);
  const dim3 grid = point_grid(a.nl[l], nlaunch(a));
  const ProbDev* probs = a.probs;
  const ProbState* cst = a.state;
  cudaError_t e;
  if (a.sk == SK_CONST)
    e = acc ? launch_pdl(a.pdl, k_jac_H<SK_CONST, true>, grid, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l,
                         a.omega, u, dst)
            : launch_pdl(a.pdl, k_jac_H<SK_CONST, false>, grid, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l,
                         a.omega, u, dst);
  else
    e = acc ? launch_pdl(a.pdl, k_jac_H<SK_FIELD, true>, grid, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l,
                         a.omega, u, dst)
            : launch_pdl(a.pdl, k_jac_H<SK_FIELD, false>, grid, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l,
                         a.omega, u, dst);
  a.prof->end(a.stream);
  return e;
}

// t = r - A e on level l into the scratch vector a.lin_t
static cudaError_t level_residual(const CycleArgs& a, int l, const float* r, const float* e, int cls) {
  a.prof->launches++;
  a.prof->begin(cls, a.stream);
  const dim3 grid = point_grid(a.nl[l], nlaunch(a));
  const ProbDev* probs = a.probs;
  const ProbState* cst = a.state;
  const cudaError_t err =
      a.sk == SK_CONST
          ? launch_pdl(a.pdl, k_lin_residual<SK_CONST>, grid, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l, r, e,
                       a.lin_t)
          : launch_pdl(a.pdl, k_lin_residual<SK_FIELD>, grid, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l, r, e,
                       a.lin_t);
  a.prof->end(a.stream);
  return err;
}

// Algorithm 1 on the levels above the tail: nu1 steps of pre-smoothing from e = 0 (e = H r,
// then e += H (r - A e)), the residual's restriction, the tail, then per level the
// prolongation and nu2 steps e += H (r - A e); the level-0 update and residual at the end
cudaError_t launch_cycle_linear(const CycleArgs& a, float rtol, int max_cycles, int parity) {
  const LevelArrays& A = *a.arrays;
  const LinMaps& M = *a.lin_maps;
  const int ls = a.lstar, np = nlaunch(a);
  const int nu1 = a.nu1 > 1 ? a.nu1 : 1, nu2 = a.nu2 > 1 ? a.nu2 : 1;
  const ProbDev* probs = a.probs;
  const ProbState* cst = a.state;
  cudaError_t e = cudaSuccess;
  auto level_r = [&](int l) -> float* { return l == 0 ? (parity ? a.r0b : a.r0a) : A.r[l]; };
  auto level_rmap = [&](int l) -> const CUtensorMap& { return l == 0 ? (parity ? M.r0b : M.r0a) : M.r[l]; };
  for (int l = 0; l < ls && e == cudaSuccess; ++l) {
    const int cls = l == 0 ? PK_DOWN0 : PK_DOWN;
    const float* r = level_r(l);
    e = smooth_H(a, l, r, level_rmap(l), A.e[l], false, cls);  // pre-smoothing from e = 0
    for (int k = 1; k < nu1 && e == cudaSuccess; ++k) {
      e = level_residual(a, l, r, A.e[l], cls);
      if (e == cudaSuccess) e = smooth_H(a, l, a.lin_t, M.t[l], A.e[l], true, cls);
    }
    if (e != cudaSuccess) break;
    a.prof->launches++;
    a.prof->begin(cls, a.stream);
    if (a.sk == SK_CONST) {
      const int nt = (a.nl[l] + HT - 1) / HT;
      e = launch_pdl(a.pdl, k_lin_restrict_tile, dim3(nt * nt, np), dim3(LTP), 0, a.stream,
                     l == 0 ? (parity ? M.rr0b : M.rr0a) : M.rr[l], M.er[l], M.rc[l], probs, a.state, a.active, l);
    } else {
      const dim3 gc = point_grid(a.nl[l + 1], np);
      e = launch_pdl(a.pdl, k_lin_restrict<SK_FIELD>, gc, dim3(PX, PY), 0, a.stream, probs, cst, a.active, l, r,
                     (const float*)A.e[l], A.r[l + 1]);
    }
    a.prof->end(a.stream);
  }
  if (e != cudaSuccess) return e;
  e = launch_tail(a);
  const bool lin = a.hk == HK_LINEAR;
  for (int l = ls - 1; l >= 0 && e == cudaSuccess; --l) {
    const int cls = l == 0 ? PK_UP0 : PK_UP;
    a.prof->launches++;
    a.prof->begin(cls, a.stream);
    // the linear smoother: prolongation, residual and the first post-smoothing step in one
    // tiled kernel whose result goes to f_l (level 0: the scratch lin_wa); Jacobi: e_l += P e_c
    float* ef = lin ? (l == 0 ? a.lin_wa : A.f[l]) : A.e[l];
    if (lin) {
      const int nt = (a.nl[l] + HT - 1) / HT;
      e = a.sk == SK_CONST
              ? launch_pdl(a.pdl, k_lin_Uptile<SK_CONST>, dim3(nt * nt, np), dim3(LTP), 0, a.stream, M.eh[l],
                           level_rmap(l), M.ec[l], probs, a.state, a.active, l, ef)
              : launch_pdl(a.pdl, k_lin_Uptile<SK_FIELD>, dim3(nt * nt, np), dim3(LTP), 0, a.stream, M.eh[l],
                           level_rmap(l), M.ec[l], probs, a.state, a.active, l, ef);
    } else {
      e = launch_pdl(a.pdl, k_lin_prolong, point_grid(a.nl[l], np), dim3(PX, PY), 0, a.stream, probs, cst, a.active,
                     l, A.e[l], (const float*)A.e[l + 1]);
    }
    a.prof->end(a.stream);
    for (int k = lin ? 1 : 0; k < nu2 && e == cudaSuccess; ++k) {  // (further) post-smoothing steps
      e = level_residual(a, l, level_r(l), ef, cls);
      if (e == cudaSuccess) e = smooth_H(a, l, a.lin_t, M.t[l], ef, true, cls);
    }
  }
  if (e != cudaSuccess || ls == 0) return e;
  // level 0: the float-float update of the iterate and its compensated residual, one
  // tiled kernel shared with the tiled path's conventions
  return launch_update_residual(a, lin ? M.e0f : M.e0, rtol, max_cycles, parity);
}

bool build_lin_maps(LinMaps& M, const LevelArrays& A, float* lin_t, float* lin_wa, int nprob, int lstar) {
  bool ok = make_map(&M.r0a, A.r[0], A.n[0], A.pitch[0], nprob, HXU, HR) &&
            make_map(&M.r0b, A.r0b, A.n[0], A.pitch[0], nprob, HXU, HR);
  int bw = 0, bh = 0;
  tile_res_box(&bw, &bh);
  ok = ok && make_map(&M.e0, A.e[0], A.n[0], A.pitch[0], nprob, bw, bh) &&
       make_map(&M.e0f, lin_wa, A.n[0], A.pitch[0], nprob, bw, bh);
  for (int l = 0; ok && l < lstar; ++l) {
    ok = make_map(&M.t[l], lin_t, A.n[l], A.pitch[l], nprob, HXU, HR) &&
         make_map(&M.eh[l], A.e[l], A.n[l], A.pitch[l], nprob, UE_X, UE_H) &&
         // the correction level l's prolongation reads: f of a batched level, the tail's e
         make_map(&M.ec[l], l + 1 < lstar ? A.f[l + 1] : A.e[l + 1], A.n[l + 1], A.pitch[l + 1], nprob, UC, UC);
    if (ok && l >= 1) ok = make_map(&M.r[l], A.r[l], A.n[l], A.pitch[l], nprob, HXU, HR);
    ok = ok && make_map(&M.er[l], A.e[l], A.n[l], A.pitch[l], nprob, RW, REH) &&
         make_map(&M.rc[l], A.r[l + 1], A.n[l + 1], A.pitch[l + 1], nprob, RCT, RCT);
    if (ok && l >= 1) ok = make_map(&M.rr[l], A.r[l], A.n[l], A.pitch[l], nprob, RW, RRH);
  }
  ok = ok && make_map(&M.rr0a, A.r[0], A.n[0], A.pitch[0], nprob, RW, RRH) &&
       make_map(&M.rr0b, A.r0b, A.n[0], A.pitch[0], nprob, RW, RRH);
  return ok;
}

// nsteps times u += H (f - A u) on level l of problem p (dense n_l x n_l vectors): the
// residual into the level's r vector, the chain through the scratch vectors
cudaError_t launch_smoother_linear(const CycleArgs& a, int p, int l, const float* f, float* u, int nsteps) {
  const int n = a.nl[l];
  const int nb = (n * n + LT - 1) / LT;
  const ProbDev* probs = a.probs;
  const float* t = a.arrays->r[l] + (size_t)p * n * a.arrays->pitch[l];
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = launch_level_residual(a, p, l, f, u);
    if (e != cudaSuccess) return e;
    const float* src = t;
    for (int k = 0; k < 4; ++k) {
      float* out = (k & 1) ? a.lin_wb : a.lin_wa;
      k_lin_conv<0><<<nb, LT, 0, a.stream>>>(probs, l, k, n, n, nullptr, nullptr, p, src, nullptr, out);
      src = out;
    }
    k_lin_conv<2><<<nb, LT, 0, a.stream>>>(probs, l, 4, n, n, nullptr, nullptr, p, src, t, u);
    a.prof->launches += 5;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_transpose_linear(float* phi, int nlev, cudaStream_t s) {
  k_lin_transpose<<<nlev, 32, 0, s>>>(phi, nlev);
  return cudaGetLastError();
}

}  // namespace mg
