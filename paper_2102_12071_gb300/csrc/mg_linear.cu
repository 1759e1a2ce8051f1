// mg_linear.cu -- the V-cycle with the shared-kernel linear smoother of Sec. 6 (eq.
// full-coarsening-smoother), for sm_103a:
//
//   H v = f_5(f_4(f_3(f_2(f_1(v))))) + f_6(v),  f_k(u)(x) = sum_t phi_k[t] u(x + d_t),
//
// six 3x3 kernels per level shared by every point (and by every problem of a context, or
// one group per problem with net_per_problem), each layer's input zero outside the grid.  The levels of side > MG_TAIL_N run as plain batched kernels over
// the pitched level arrays, one thread per point with the neighbours through L1 (a pass of
// the chain reads and writes 8 bytes per point; the level arrays of the batch are mostly
// L2-resident at the sizes the paper uses); the levels below run in the one-CTA tail
// (mg_tail.cuh), which holds the chain in shared memory.  The level-0 update and the
// compensated residual with the stopping test follow the same conventions as the tiled
// path (iterate and residual alternate between two arrays by cycle parity).
#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_ops.cuh"
#include "mg_reduce.cuh"
#include "mg_tma.cuh"

namespace mg {

constexpr int LT = 256;  // threads per CTA of the point kernels
constexpr int TB = 32;   // tile side of the residual/norm kernel (matches the partial slots)

// problem of this CTA (-1: none) and the offset of its slice of a [nprob][n][pitch] array
__device__ __forceinline__ int lin_problem(const ProbState* state, const int* act, int pfix) {
  if (pfix >= 0) return pfix;
  const int p = act ? act[blockIdx.y] : blockIdx.y;
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
  const int p = lin_problem(state, act, pfix);
  if (p < 0 || q >= n * n) return;
  const size_t off = pfix >= 0 ? 0 : (size_t)p * n * pitch;
  const int i = q / n, j = q % n;
  const size_t o = off + (size_t)i * pitch + j;
  float h = conv_at(w, src + off, pitch, n, i, j);
  if (MODE) h += conv_at(w6, src2 + off, pitch, n, i, j);
  dst[o] = MODE == 2 ? dst[o] + h : h;
}

// r_{l+1} = P^T (r - A e), one thread per coarse point: the residual on the 3 x 3 fine
// points of its restriction stencil (fine 2I+1+d, all inside the grid) from e's 5 x 5
// neighbourhood, then the restriction of Sec. 6.1 in the tile kernels' summation order.
template <int SK>
__global__ void __launch_bounds__(LT) k_lin_restrict(const ProbDev* __restrict__ probs,
                                                     const ProbState* __restrict__ state, const int* __restrict__ act,
                                                     int l, const float* r, const float* e, float* rc) {
  pdl_trigger();
  const int Q = blockIdx.x * LT + threadIdx.x;
  pdl_wait();
  const int p = lin_problem(state, act, -1);
  if (p < 0) return;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, pitch = L.pitch, nc = probs[p].lv[l + 1].n, pc = probs[p].lv[l + 1].pitch;
  if (Q >= nc * nc) return;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  const int I = Q / nc, J = Q % nc;
  const size_t off = (size_t)p * n * pitch;
  const float* rp = r + off;
  const float* ep = e + off;
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

// e_l += P e_{l+1} (bilinear, Sec. 6.1), one thread per fine point, coarse values zero
// outside the coarse grid; the arithmetic of prolong_at
__global__ void __launch_bounds__(LT) k_lin_prolong(const ProbDev* __restrict__ probs,
                                                    const ProbState* __restrict__ state, const int* __restrict__ act,
                                                    int l, float* e, const float* ec) {
  pdl_trigger();
  const int q = blockIdx.x * LT + threadIdx.x;
  pdl_wait();
  const int p = lin_problem(state, act, -1);
  if (p < 0) return;
  const int n = probs[p].lv[l].n, pitch = probs[p].lv[l].pitch;
  const int nc = probs[p].lv[l + 1].n, pc = probs[p].lv[l + 1].pitch;
  if (q >= n * n) return;
  const int i = q / n, j = q % n;
  const float* c = ec + (size_t)p * nc * pc;
  const int Ia = (i - 1) >> 1, Ja = (j - 1) >> 1;
  const float b00 = tap_at(c, pc, nc, Ia, Ja), b01 = tap_at(c, pc, nc, Ia, Ja + 1);
  const float b10 = tap_at(c, pc, nc, Ia + 1, Ja), b11 = tap_at(c, pc, nc, Ia + 1, Ja + 1);
  float v;
  if (i & 1) v = (j & 1) ? b00 : 0.5f * (b00 + b01);
  else v = (j & 1) ? 0.5f * (b00 + b10) : 0.25f * ((b00 + b01) + (b10 + b11));
  e[(size_t)p * n * pitch + (size_t)i * pitch + j] += v;
}

// t = r - A e on one level
template <int SK>
__global__ void __launch_bounds__(LT) k_lin_residual(const ProbDev* __restrict__ probs,
                                                     const ProbState* __restrict__ state, const int* __restrict__ act,
                                                     int l, const float* r, const float* e, float* t) {
  pdl_trigger();
  const int q = blockIdx.x * LT + threadIdx.x;
  pdl_wait();
  const int p = lin_problem(state, act, -1);
  if (p < 0) return;
  const LevelDev L = probs[p].lv[l];
  const int n = L.n, pitch = L.pitch;
  if (q >= n * n) return;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  const int i = q / n, j = q % n;
  const size_t off = (size_t)p * n * pitch, o = off + (size_t)i * pitch + j;
  t[o] = r[o] - apply_A_at<SK>(L, s, e + off, pitch, i, j);
}

// x_out = x_in + e_0 in float-float (the update of the fused level-0 kernel)
__global__ void __launch_bounds__(LT) k_lin_xupdate(const ProbDev* __restrict__ probs,
                                                    const ProbState* __restrict__ state, const int* __restrict__ act,
                                                    const float* e, const float* xh_in, const float* xl_in,
                                                    float* xh_out, float* xl_out) {
  pdl_trigger();
  const int q = blockIdx.x * LT + threadIdx.x;
  pdl_wait();
  const int p = lin_problem(state, act, -1);
  if (p < 0) return;
  const int n = probs[p].lv[0].n, pitch = probs[p].lv[0].pitch;
  if (q >= n * n) return;
  const size_t o = (size_t)p * n * pitch + (size_t)(q / n) * pitch + q % n;
  float hi = xh_in[o], lo = xl_in[o], sum, err;
  two_sum(hi, e[o], sum, err);
  err += lo;
  fast_two_sum(sum, err, hi, lo);
  xh_out[o] = hi;
  xl_out[o] = lo;
}

// r = b - A (x_hi + x_lo) (Dot2, the taps in index order), ||r||^2 per 32 x 32 tile into
// the partial slots and, in the last CTA of a problem, the stopping test
template <int SK>
__global__ void __launch_bounds__(LT) k_lin_residual0(const ProbDev* __restrict__ probs, ProbState* __restrict__ state,
                                                      const int* __restrict__ act, float* __restrict__ partials,
                                                      int ntiles_max, float rtol, int max_cycles, const float* xh,
                                                      const float* xl, const float* b, float* rout) {
  pdl_trigger();
  pdl_wait();
  const int p = lin_problem(state, act, -1);
  if (p < 0) return;
  const LevelDev L = probs[p].lv[0];
  const int n = L.n, pitch = L.pitch;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx, tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  float s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = (SK == SK_CONST) ? L.s[k] : 0.f;
  const size_t off = (size_t)p * n * pitch;
  const float *xh_p = xh + off, *xl_p = xl + off;
  const int j = C0 + (threadIdx.x & 31);
  float acc = 0.f;
  for (int k = 0; k < TB / (LT / 32); ++k) {
    const int i = R0 + (threadIdx.x >> 5) * (TB / (LT / 32)) + k;
    if (i >= n || j >= n) continue;
    const size_t o = (size_t)i * pitch + j;
    float a[9];
    if (SK == SK_CONST) {
#pragma unroll
      for (int t = 0; t < 9; ++t) a[t] = s[t];
    } else {
      const size_t nn = (size_t)n * n, qq = (size_t)i * n + j;
#pragma unroll
      for (int t = 0; t < 9; ++t) a[t] = __ldg(L.st + t * nn + qq);
    }
    float hi = b[off + o], lo = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int ii = i + t / 3 - 1, jj = j + t % 3 - 1;
      if ((unsigned)ii < (unsigned)n && (unsigned)jj < (unsigned)n) {
        const size_t on = (size_t)ii * pitch + jj;
        dot2_sub(a[t], xh_p[on], xl_p[on], hi, lo);
      }
    }
    const float rv = hi + lo;
    rout[off + o] = rv;
    acc = fmaf(rv, rv, acc);
  }
  float rhi, rlo;
  if (block_partial_and_last<LT>(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, rhi, rlo)) {
    if (threadIdx.x == 0) decide(state[p], rhi, rlo, rtol, max_cycles);
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

// one application of H on level l over the launch set: dst (=, or += with acc) H u,
// through the scratch vectors a.lin_wa / a.lin_wb
static cudaError_t lin_H(const CycleArgs& a, int l, const float* u, float* dst, bool acc, int cls) {
  const int n = a.nl[l], pitch = a.arrays->pitch[l];
  const dim3 grid((n * n + LT - 1) / LT, nlaunch(a));
  const ProbDev* probs = a.probs;
  const float* src = u;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
    float* out = (k & 1) ? a.lin_wb : a.lin_wa;
    a.prof->launches++;
    a.prof->begin(cls, a.stream);
    e = launch_pdl(a.pdl, k_lin_conv<0>, grid, dim3(LT), 0, a.stream, probs, l, k, n, pitch, (const ProbState*)a.state,
                   a.active, -1, src, (const float*)nullptr, out);
    a.prof->end(a.stream);
    src = out;
  }
  if (e != cudaSuccess) return e;
  a.prof->launches++;
  a.prof->begin(cls, a.stream);
  e = acc ? launch_pdl(a.pdl, k_lin_conv<2>, grid, dim3(LT), 0, a.stream, probs, l, 4, n, pitch,
                       (const ProbState*)a.state, a.active, -1, src, u, dst)
          : launch_pdl(a.pdl, k_lin_conv<1>, grid, dim3(LT), 0, a.stream, probs, l, 4, n, pitch,
                       (const ProbState*)a.state, a.active, -1, src, u, dst);
  a.prof->end(a.stream);
  return e;
}

cudaError_t launch_cycle_linear(const CycleArgs& a, float rtol, int max_cycles, int parity) {
  const LevelArrays& A = *a.arrays;
  const int ls = a.lstar, np = nlaunch(a);
  const ProbDev* probs = a.probs;
  const ProbState* cst = a.state;
  cudaError_t e = cudaSuccess;
  auto level_r = [&](int l) -> float* { return l == 0 ? (parity ? a.r0b : a.r0a) : A.r[l]; };
  for (int l = 0; l < ls && e == cudaSuccess; ++l) {
    const int cls = l == 0 ? PK_DOWN0 : PK_DOWN;
    e = lin_H(a, l, level_r(l), A.e[l], false, cls);  // pre-smoothing from e = 0
    if (e != cudaSuccess) break;
    const int nc = a.nl[l + 1];
    const dim3 grid((nc * nc + LT - 1) / LT, np);
    a.prof->launches++;
    a.prof->begin(cls, a.stream);
    e = a.sk == SK_CONST
            ? launch_pdl(a.pdl, k_lin_restrict<SK_CONST>, grid, dim3(LT), 0, a.stream, probs, cst, a.active, l,
                         (const float*)level_r(l), (const float*)A.e[l], A.r[l + 1])
            : launch_pdl(a.pdl, k_lin_restrict<SK_FIELD>, grid, dim3(LT), 0, a.stream, probs, cst, a.active, l,
                         (const float*)level_r(l), (const float*)A.e[l], A.r[l + 1]);
    a.prof->end(a.stream);
  }
  if (e != cudaSuccess) return e;
  e = launch_tail(a);
  for (int l = ls - 1; l >= 0 && e == cudaSuccess; --l) {
    const int cls = l == 0 ? PK_UP0 : PK_UP;
    const int n = a.nl[l];
    const dim3 grid((n * n + LT - 1) / LT, np);
    a.prof->launches += 2;
    a.prof->begin(cls, a.stream);
    e = launch_pdl(a.pdl, k_lin_prolong, grid, dim3(LT), 0, a.stream, probs, cst, a.active, l, A.e[l],
                   (const float*)A.e[l + 1]);
    a.prof->end(a.stream);
    if (e != cudaSuccess) break;
    a.prof->begin(cls, a.stream);
    e = a.sk == SK_CONST
            ? launch_pdl(a.pdl, k_lin_residual<SK_CONST>, grid, dim3(LT), 0, a.stream, probs, cst, a.active, l,
                         (const float*)level_r(l), (const float*)A.e[l], a.lin_t)
            : launch_pdl(a.pdl, k_lin_residual<SK_FIELD>, grid, dim3(LT), 0, a.stream, probs, cst, a.active, l,
                         (const float*)level_r(l), (const float*)A.e[l], a.lin_t);
    a.prof->end(a.stream);
    if (e != cudaSuccess) break;
    e = lin_H(a, l, a.lin_t, A.e[l], true, cls);  // post-smoothing
  }
  if (e != cudaSuccess || ls == 0) return e;
  // level 0: the float-float update of the iterate, then its compensated residual
  const int n = a.n0;
  const float* xh_in = parity ? a.xh0b : a.xh0;
  const float* xl_in = parity ? a.xl0b : a.xl0;
  float* xh_out = parity ? a.xh0 : a.xh0b;
  float* xl_out = parity ? a.xl0 : a.xl0b;
  float* rnew = parity ? a.r0a : a.r0b;
  a.prof->launches += 2;
  a.prof->begin(PK_UP0, a.stream);
  e = launch_pdl(a.pdl, k_lin_xupdate, dim3((n * n + LT - 1) / LT, np), dim3(LT), 0, a.stream, probs, cst, a.active,
                 (const float*)A.e[0], xh_in, xl_in, xh_out, xl_out);
  a.prof->end(a.stream);
  if (e != cudaSuccess) return e;
  const int nt = (n + TB - 1) / TB;
  a.prof->begin(PK_UP0, a.stream);
  e = a.sk == SK_CONST
          ? launch_pdl(a.pdl, k_lin_residual0<SK_CONST>, dim3(nt * nt, np), dim3(LT), 0, a.stream, probs, a.state,
                       a.active, a.partials, a.ntiles_max, rtol, max_cycles, (const float*)xh_out,
                       (const float*)xl_out, a.b0, rnew)
          : launch_pdl(a.pdl, k_lin_residual0<SK_FIELD>, dim3(nt * nt, np), dim3(LT), 0, a.stream, probs, a.state,
                       a.active, a.partials, a.ntiles_max, rtol, max_cycles, (const float*)xh_out,
                       (const float*)xl_out, a.b0, rnew);
  a.prof->end(a.stream);
  return e;
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
