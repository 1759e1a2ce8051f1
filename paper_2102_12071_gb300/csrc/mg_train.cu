// mg_train.cu -- the convergence-theory training loss and its adjoint (Sec. 3.2).
//
// For problem b and random vector z_bj (Thm. sbound), with S = I - H A and the two-grid
// coarse correction C = I - P (P^T A P)^{-1} P^T A (eq. twogrid, one pre- and one
// post-smoothing step):
//   e0 = z,  v0 = A e0,  e1 = e0 - H v0,  e2 = C e1,  v2 = A e2,  e3 = e2 - H v2,
//   loss = (1/B) sum_b (1/Z) sum_j ||e3||^2 / n^2.
// Adjoint: g3 = 2 e3 / (n^2 Z B); dW_p[k] -= g3(p) v2(p+d_k); g2 = g3 - A H^T g3;
//          g1 = g2 - A P (P^T A P)^{-1} P^T g2; dW_p[k] -= g1(p) v0(p+d_k);
// then dW -> d(params) through the network (mg_net.cu).
// After k cycles (E = S C S, loss = ... ||E^k z||^2): the forward keeps A e and A (C S e)
// of every cycle, or with checkpointing only each cycle's input e and recomputes the two
// products when the adjoint reaches that cycle; the adjoint runs the cycles in reverse,
// adds both dW terms of each, and passes E^T g = S^T C^T S^T g to the cycle before.
//
// All problems of a batch share n, so every kernel runs over (problem, vector, point) in
// one launch; the data of a 64 x 32 batch at 63^2 (~16 MB per vector set) stays in L2.
// The two-grid coarse operator is solved exactly in FP64 by a banded Cholesky factor
// (bandwidth n_c + 1 <= 32): this is the coarsest-level direct solve of the two-grid
// hierarchy, the one place FP64 is used.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "mg_internal.h"
#include "mgcnn.h"

namespace mg {

constexpr int TT = 256;

__device__ __forceinline__ float appA(const float* __restrict__ st, const float* __restrict__ v, int n, int i, int j) {
  const size_t nn = (size_t)n * n;
  const int q = i * n + j;
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
    if (in_grid(ii, jj, n)) acc = fmaf(st[k * nn + q], v[ii * n + jj], acc);
  }
  return acc;
}

// (H^T v)(y) = sum_k W_{y - d_k}[k] v(y - d_k)
__device__ __forceinline__ float appHT(const float* __restrict__ W, const float* __restrict__ v, int n, int i, int j) {
  const size_t nn = (size_t)n * n;
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ii = i - (k / 3 - 1), jj = j - (k % 3 - 1);
    if (in_grid(ii, jj, n)) acc = fmaf(W[k * nn + ii * n + jj], v[ii * n + jj], acc);
  }
  return acc;
}

struct TrainDims {
  int n, nc, B, Z, w;  // w = band width of the coarse factor
  size_t nn, nnc;
};

// vector index: blockIdx.y = b*Z + j; points: blockIdx.x * TT + threadIdx.x
#define T_PROLOGUE                                           \
  const int vec = blockIdx.y, b = vec / D.Z;                 \
  const int q = blockIdx.x * TT + threadIdx.x;               \
  if (q >= (int)D.nn) return;                                \
  const int i = q / D.n, j = q % D.n;                        \
  const size_t off = (size_t)vec * D.nn;                     \
  const float* st = fields + (size_t)b * 9 * D.nn;           \
  (void)i; (void)j; (void)st;

// the same for kernels that touch no stencil
#define T_PROLOGUE_V                                         \
  const int vec = blockIdx.y;                                \
  const int q = blockIdx.x * TT + threadIdx.x;               \
  if (q >= (int)D.nn) return;                                \
  const int i = q / D.n, j = q % D.n;                        \
  const size_t off = (size_t)vec * D.nn;

// out = A in
__global__ void k_t_applyA(TrainDims D, const float* __restrict__ fields, const float* __restrict__ in,
                           float* __restrict__ out) {
  T_PROLOGUE
  out[off + q] = appA(st, in + off, D.n, i, j);
}

// out = x - H v
__global__ void k_t_xmHv(TrainDims D, const float* __restrict__ fields, const float* __restrict__ Wall,
                         const float* __restrict__ x, const float* __restrict__ v, float* __restrict__ out) {
  T_PROLOGUE
  const float* W = Wall + (size_t)b * 9 * D.nn;
  const float* vv = v + off;
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
    if (in_grid(ii, jj, D.n)) acc = fmaf(W[k * D.nn + q], vv[ii * D.n + jj], acc);
  }
  out[off + q] = x[off + q] - acc;
}

// out = x - A v
__global__ void k_t_xmAv(TrainDims D, const float* __restrict__ fields, const float* __restrict__ x,
                         const float* __restrict__ v, float* __restrict__ out) {
  T_PROLOGUE
  out[off + q] = x[off + q] - appA(st, v + off, D.n, i, j);
}

// out = H^T v
__global__ void k_t_HT(TrainDims D, const float* __restrict__ fields, const float* __restrict__ Wall,
                       const float* __restrict__ v, float* __restrict__ out) {
  T_PROLOGUE
  out[off + q] = appHT(Wall + (size_t)b * 9 * D.nn, v + off, D.n, i, j);
}

// coarse rc = P^T (A v) if withA, else P^T v  (one thread per coarse point)
__global__ void k_t_restrict(TrainDims D, const float* __restrict__ fields, const float* __restrict__ v, int withA,
                             float* __restrict__ rc) {
  const int vec = blockIdx.y, b = vec / D.Z;
  const int Q = blockIdx.x * TT + threadIdx.x;
  if (Q >= (int)D.nnc) return;
  const int I = Q / D.nc, J = Q % D.nc;
  const float* st = fields + (size_t)b * 9 * D.nn;
  const float* vv = v + (size_t)vec * D.nn;
  float acc = 0.f;
  for (int di = -1; di <= 1; ++di)
    for (int dj = -1; dj <= 1; ++dj) {
      const int fi = 2 * I + 1 + di, fj = 2 * J + 1 + dj;
      const float val = withA ? appA(st, vv, D.n, fi, fj) : vv[fi * D.n + fj];
      acc = fmaf((di ? 0.5f : 1.f) * (dj ? 0.5f : 1.f), val, acc);
    }
  rc[(size_t)vec * D.nnc + Q] = acc;
}

// out = x - P xc  (P bilinear)
__global__ void k_t_xmP(TrainDims D, const float* __restrict__ x, const float* __restrict__ xc,
                        float* __restrict__ out) {
  const int vec = blockIdx.y;
  const int q = blockIdx.x * TT + threadIdx.x;
  if (q >= (int)D.nn) return;
  const int i = q / D.n, j = q % D.n;
  const float* c = xc + (size_t)vec * D.nnc;
  float v = 0.f;
  for (int di = -1; di <= 1; ++di)
    for (int dj = -1; dj <= 1; ++dj) {
      const int fi = i + di, fj = j + dj;
      if ((fi & 1) && (fj & 1)) {
        const int I = (fi - 1) >> 1, J = (fj - 1) >> 1;
        if (in_grid(I, J, D.nc)) v += (di ? 0.5f : 1.f) * (dj ? 0.5f : 1.f) * c[I * D.nc + J];
      }
    }
  out[(size_t)vec * D.nn + q] = x[(size_t)vec * D.nn + q] - v;
}

// per-vector sum of squares (one CTA per vector) and g3 = scale * e3 (g3 may be e3: in place)
__global__ void k_t_loss(TrainDims D, const float* e3, float scale, float* g3, float* __restrict__ partial) {
  const int vec = blockIdx.x;
  const float* e = e3 + (size_t)vec * D.nn;
  float* g = g3 + (size_t)vec * D.nn;
  float acc = 0.f;
  for (int q = threadIdx.x; q < (int)D.nn; q += TT) {
    const float v = e[q];
    acc = fmaf(v, v, acc);
    g[q] = scale * v;
  }
  __shared__ float ws[TT / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int k = 0; k < TT / 32; ++k) s += ws[k];
    partial[vec] = s;
  }
}

__global__ void k_t_loss_total(const float* __restrict__ partial, int nvecs, float scale, float* __restrict__ loss) {
  float hi = 0.f, lo = 0.f;
  for (int t = threadIdx.x; t < nvecs; t += 32) ff_add(hi, lo, partial[t], 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, oh, ol);
  }
  if (threadIdx.x == 0) *loss = scale * (hi + lo);
}

// dW_p[k] = -sum_j ( g3_j(p) v2_j(p+d_k) + g1_j(p) v0_j(p+d_k) )   (one thread per (b, p))
__global__ void k_t_dW(TrainDims D, const float* __restrict__ g3, const float* __restrict__ v2,
                       const float* __restrict__ g1, const float* __restrict__ v0, float* __restrict__ dW,
                       int accumulate) {
  const int b = blockIdx.y;
  const int q = blockIdx.x * TT + threadIdx.x;
  if (q >= (int)D.nn) return;
  const int i = q / D.n, j = q % D.n;
  float acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.f;
  for (int z = 0; z < D.Z; ++z) {
    const size_t off = ((size_t)b * D.Z + z) * D.nn;
    const float a3 = g3[off + q], a1 = g1[off + q];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
      if (in_grid(ii, jj, D.n)) {
        const int r = ii * D.n + jj;
        acc[k] = fmaf(a3, v2[off + r], acc[k]);
        acc[k] = fmaf(a1, v0[off + r], acc[k]);
      }
    }
  }
  float* out = dW + (size_t)b * 9 * D.nn;
#pragma unroll
  for (int k = 0; k < 9; ++k) out[k * D.nn + q] = accumulate ? out[k * D.nn + q] - acc[k] : -acc[k];
}

// ------------------------------------------------- the three-kernel stack (MG_NET_CONV3)
// H = K3 K2 K1, kernel k (0..2) of problem b at Wall + (27 b + 9 k) nn, tap t at + t nn.
__device__ __forceinline__ const float* t3_kernel(const TrainDims& D, const float* Wall, int b, int k) {
  return Wall + ((size_t)b * 27 + 9 * k) * D.nn;
}

// out = K_k in, or out = x - K_k in when x is given
__global__ void k_t3_conv(TrainDims D, const float* __restrict__ Wall, int k, const float* __restrict__ x,
                          const float* __restrict__ in, float* __restrict__ out) {
  T_PROLOGUE_V
  const float* W = t3_kernel(D, Wall, vec / D.Z, k);
  const float* v = in + off;
  float acc = 0.f;
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int ii = i + t / 3 - 1, jj = j + t % 3 - 1;
    if (in_grid(ii, jj, D.n)) acc = fmaf(W[t * D.nn + q], v[ii * D.n + jj], acc);
  }
  out[off + q] = x ? x[off + q] - acc : acc;
}

// out = K_k^T in
__global__ void k_t3_convT(TrainDims D, const float* __restrict__ Wall, int k, const float* __restrict__ in,
                           float* __restrict__ out) {
  T_PROLOGUE_V
  out[off + q] = appHT(t3_kernel(D, Wall, vec / D.Z, k), in + off, D.n, i, j);
}

// dW[9k + t](p) -= sum_j g_j(p) u_j(p + d_t): the gradient of a term x - K_k u with output
// gradient g (one thread per (b, p); dW is cleared before the adjoint)
__global__ void k_t3_dW(TrainDims D, const float* __restrict__ g, const float* __restrict__ u,
                        float* __restrict__ dW, int k) {
  const int b = blockIdx.y;
  const int q = blockIdx.x * TT + threadIdx.x;
  if (q >= (int)D.nn) return;
  const int i = q / D.n, j = q % D.n;
  float acc[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) acc[t] = 0.f;
  for (int z = 0; z < D.Z; ++z) {
    const size_t off = ((size_t)b * D.Z + z) * D.nn;
    const float gv = g[off + q];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int ii = i + t / 3 - 1, jj = j + t % 3 - 1;
      if (in_grid(ii, jj, D.n)) acc[t] = fmaf(gv, u[off + ii * D.n + jj], acc[t]);
    }
  }
  float* out = dW + ((size_t)b * 27 + 9 * k) * D.nn;
#pragma unroll
  for (int t = 0; t < 9; ++t) out[t * D.nn + q] -= acc[t];
}

// ---------------------------------------------------------------- coarse solve
// Banded Cholesky of the Galerkin coarse operator, right-looking, one CTA per problem.
// band[(r)*(w+1) + d] holds L(r, r-d), d = 0..w.  A(r, r-d) comes from the coarse field.
__global__ void k_t_band_factor(TrainDims D, const float* __restrict__ cfields, double* __restrict__ band,
                                int* __restrict__ fail) {
  const int b = blockIdx.x;
  const int nc = D.nc, m = nc * nc, w = D.w, ld = w + 1;
  const float* cst = cfields + (size_t)b * 9 * D.nnc;
  double* L = band + (size_t)b * m * ld;
  // fill the lower band of A: row r = (I, J), column c = r - d
  for (int t = threadIdx.x; t < m * ld; t += blockDim.x) {
    const int r = t / ld, d = t % ld;
    const int c = r - d;
    double v = 0.0;
    if (c >= 0) {
      const int I = r / nc, J = r % nc, I2 = c / nc, J2 = c % nc;
      const int di = I2 - I, dj = J2 - J;
      if (di >= -1 && di <= 1 && dj >= -1 && dj <= 1) v = (double)cst[(3 * (di + 1) + dj + 1) * D.nnc + r];
    }
    L[t] = v;
  }
  __syncthreads();
  __shared__ double piv;
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      const double d = L[(size_t)k * ld];
      if (!(d > 0.0)) atomicExch(fail, 1);
      piv = d > 0.0 ? sqrt(d) : 1.0;
      L[(size_t)k * ld] = piv;
    }
    __syncthreads();
    // column k below the diagonal: rows k+1 .. k+w
    for (int t = threadIdx.x; t < w; t += blockDim.x) {
      const int r = k + 1 + t;
      if (r < m) L[(size_t)r * ld + (r - k)] /= piv;
    }
    __syncthreads();
    // trailing update: A(r, c) -= L(r, k) L(c, k) for k < c <= r <= k+w
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      const int r = k + 1 + t / w, c = k + 1 + t % w;
      if (c <= r && r < m) L[(size_t)r * ld + (r - c)] -= L[(size_t)r * ld + (r - k)] * L[(size_t)c * ld + (c - k)];
    }
    __syncthreads();
  }
}

// After factorisation: the diagonal slot holds 1/L(i,i) and ut[(i)*(w+1) + d] = L(i+d, i)
// (the band transposed, so the backward sweep reads rows contiguously).
__global__ void k_t_band_finish(TrainDims D, double* __restrict__ band, double* __restrict__ ut) {
  const int b = blockIdx.y;
  const int m = D.nc * D.nc, ld = D.w + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * ld) return;
  const int i = t / ld, d = t % ld;
  double* L = band + (size_t)b * m * ld;
  double* U = ut + (size_t)b * m * ld;
  U[t] = (d > 0 && i + d < m) ? L[(size_t)(i + d) * ld + d] : (d == 0 ? 1.0 / L[(size_t)i * ld] : 0.0);
}

__global__ void k_t_band_invdiag(TrainDims D, double* __restrict__ band) {
  const int b = blockIdx.y;
  const int m = D.nc * D.nc, ld = D.w + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double* L = band + (size_t)b * m * ld;
  L[(size_t)i * ld] = 1.0 / L[(size_t)i * ld];
}

// x = A_c^{-1} rhs, one warp per right-hand side: forward substitution with L, then
// backward substitution with L^T, FP64 throughout, right-looking: lane t keeps the pending
// sum of the row t below (above) the current one, so a step is one product for the current
// unknown, one multiply-add per lane with its column of L, and a one-lane shift of the
// window, whose new last row takes its own update when the band reaches it (w = 32).  Each
// step's band entries are loaded one step ahead.
__global__ void k_t_band_solve(TrainDims D, const double* __restrict__ band, const double* __restrict__ ut,
                               const float* __restrict__ rhs, double* __restrict__ ybuf, float* __restrict__ x,
                               int nvecs) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nvecs) return;
  const int b = warp / D.Z;
  const int m = D.nc * D.nc, w = D.w, ld = w + 1;
  const double* L = band + (size_t)b * m * ld;  // L(r, r-d) at r*ld + d, 1/L(r,r) at r*ld
  const double* U = ut + (size_t)b * m * ld;    // L(i+d, i) at i*ld + d, 1/L(i,i) at i*ld
  const float* r = rhs + (size_t)warp * D.nnc;
  double* y = ybuf + (size_t)warp * m;
  float* out = x + (size_t)warp * D.nnc;
  const bool upd = lane >= 1 && lane <= w;
  const bool edge = w == 32;
  // forward: lane t holds the pending sum of row i + t
  double acc = lane < m ? (double)r[lane] : 0.0;
  double cn = upd ? U[lane] : 0.0, dn = U[0], en = edge ? U[32] : 0.0;
  double rn = 32 < m ? (double)r[32] : 0.0;
  for (int i = 0; i < m; ++i) {
    const double c = cn, dinv = dn, ce = en, rin = rn;
    if (i + 1 < m) {
      const double* Ui = U + (size_t)(i + 1) * ld;
      cn = upd ? Ui[lane] : 0.0;
      dn = Ui[0];
      en = edge ? Ui[32] : 0.0;
      rn = i + 33 < m ? (double)r[i + 33] : 0.0;
    }
    const double yi = __shfl_sync(0xffffffffu, acc, 0) * dinv;
    if (lane == 0) y[i] = yi;
    acc = fma(-c, yi, acc);
    const double enter = i + 32 < m ? fma(-ce, yi, rin) : 0.0;
    acc = __shfl_down_sync(0xffffffffu, acc, 1);
    if (lane == 31) acc = enter;
  }
  __syncwarp();
  // backward: lane t holds the pending sum of row i - t
  acc = lane < m ? y[m - 1 - lane] : 0.0;
  {
    const double* Li = L + (size_t)(m - 1) * ld;
    cn = upd ? Li[lane] : 0.0;
    dn = Li[0];
    en = edge ? Li[32] : 0.0;
  }
  double yn = m - 33 >= 0 ? y[m - 33] : 0.0;
  for (int i = m - 1; i >= 0; --i) {
    const double c = cn, dinv = dn, ce = en, yin = yn;
    if (i > 0) {
      const double* Li = L + (size_t)(i - 1) * ld;
      cn = upd ? Li[lane] : 0.0;
      dn = Li[0];
      en = edge ? Li[32] : 0.0;
      yn = i - 33 >= 0 ? y[i - 33] : 0.0;
    }
    const double xi = __shfl_sync(0xffffffffu, acc, 0) * dinv;
    if (lane == 0) out[i] = (float)xi;
    acc = fma(-c, xi, acc);
    const double enter = i - 32 >= 0 ? fma(-ce, xi, yin) : 0.0;
    acc = __shfl_down_sync(0xffffffffu, acc, 1);
    if (lane == 31) acc = enter;
  }
}

// ------------------------------------------------- the shared-kernel linear smoother
// H v = f5(f4(f3(f2(f1 v)))) + f6 v (Sec. 6, eq. full-coarsening-smoother), one 3x3
// kernel per layer shared by every point of every vector, each layer's input zero outside
// the grid.  Forward: four plain passes and x - (f5 w4 + f6 v).  Adjoint of one
// application e_out = x - H v with output gradient g: the passes recomputed from v, then
// back through the chain (transposed passes), the kernel gradients as correlations
// sum_x lambda(x) w(x + d_t) reduced in a fixed order, and H^T g for the state adjoint.

// sum_t w[t] v(i + di_t, j + dj_t) on one dense n x n vector, centre tap first
__device__ __forceinline__ float tl_conv_at(const float* w, const float* v, int n, int i, int j) {
  float acc = w[4] * v[i * n + j];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    if (t == 4) continue;
    const int ii = i + t / 3 - 1, jj = j + t % 3 - 1;
    if (in_grid(ii, jj, n)) acc = fmaf(w[t], v[ii * n + jj], acc);
  }
  return acc;
}

// sum_t w[t] v(i - di_t, j - dj_t): the transposed pass
__device__ __forceinline__ float tl_convT_at(const float* w, const float* v, int n, int i, int j) {
  float acc = w[4] * v[i * n + j];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    if (t == 4) continue;
    const int ii = i - (t / 3 - 1), jj = j - (t % 3 - 1);
    if (in_grid(ii, jj, n)) acc = fmaf(w[t], v[ii * n + jj], acc);
  }
  return acc;
}

// out = f(in), kernel w (9 floats), every vector
__global__ void k_tl_conv(TrainDims D, const float* __restrict__ w, const float* __restrict__ in,
                          float* __restrict__ out) {
  T_PROLOGUE_V
  out[off + q] = tl_conv_at(w, in + off, D.n, i, j);
}

// out = f^T(in)
__global__ void k_tl_convT(TrainDims D, const float* __restrict__ w, const float* __restrict__ in,
                           float* __restrict__ out) {
  T_PROLOGUE_V
  out[off + q] = tl_convT_at(w, in + off, D.n, i, j);
}

// out = x - (f5(w4) + f6(v))
__global__ void k_tl_xmH(TrainDims D, const float* __restrict__ phi, const float* __restrict__ x,
                         const float* __restrict__ w4, const float* __restrict__ v, float* __restrict__ out) {
  T_PROLOGUE_V
  const float h = tl_conv_at(phi + 36, w4 + off, D.n, i, j) + tl_conv_at(phi + 45, v + off, D.n, i, j);
  out[off + q] = x[off + q] - h;
}

// out = H^T g = f1^T(l1) + f6^T(g)
__global__ void k_tl_HT(TrainDims D, const float* __restrict__ phi, const float* __restrict__ l1,
                        const float* __restrict__ g, float* __restrict__ out) {
  T_PROLOGUE_V
  out[off + q] = tl_convT_at(phi, l1 + off, D.n, i, j) + tl_convT_at(phi + 45, g + off, D.n, i, j);
}

// partial[(vec * gridDim.x + block) * 9 + t] = sum over the block's points x of g(x) u(x + d_t)
__global__ void k_tl_corr(TrainDims D, const float* __restrict__ g, const float* __restrict__ u,
                          float* __restrict__ partial) {
  const int vec = blockIdx.y;
  const int q = blockIdx.x * TT + threadIdx.x;
  float c[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) c[t] = 0.f;
  if (q < (int)D.nn) {
    const int i = q / D.n, j = q % D.n;
    const size_t off = (size_t)vec * D.nn;
    const float gv = g[off + q];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int ii = i + t / 3 - 1, jj = j + t % 3 - 1;
      if (in_grid(ii, jj, D.n)) c[t] = gv * u[off + ii * D.n + jj];
    }
  }
  __shared__ float ws[9][TT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const float v = warp_sum(c[t]);
    if (lane == 0) ws[t][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    float s = 0.f;
    for (int k = 0; k < TT / 32; ++k) s += ws[threadIdx.x][k];
    partial[((size_t)vec * gridDim.x + blockIdx.x) * 9 + threadIdx.x] = s;
  }
}

// grad[slot * 9 + t] -= sum of the count partials of tap t (float-float, fixed order); 9 CTAs
__global__ void k_tl_reduce(const float* __restrict__ partial, int count, float* __restrict__ grad, int slot) {
  const int t = blockIdx.x;
  float hi = 0.f, lo = 0.f;
  for (int k = threadIdx.x; k < count; k += TT) ff_add(hi, lo, partial[(size_t)k * 9 + t], 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, oh, ol);
  }
  __shared__ float sh[TT / 32], sl[TT / 32];
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = hi;
    sl[threadIdx.x >> 5] = lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float h = 0.f, l = 0.f;
    for (int k = 0; k < TT / 32; ++k) ff_add(h, l, sh[k], sl[k]);
    grad[slot * 9 + t] -= h + l;
  }
}

// constant stencils expanded to truncated fields
__global__ void k_t_const_field(TrainDims D, const float* __restrict__ s9, float* __restrict__ fields) {
  const int b = blockIdx.y;
  const int q = blockIdx.x * TT + threadIdx.x;
  if (q >= (int)D.nn) return;
  const int i = q / D.n, j = q % D.n;
  const float* s = s9 + 9 * b;
  float* st = fields + (size_t)b * 9 * D.nn;
#pragma unroll
  for (int k = 0; k < 9; ++k) st[k * D.nn + q] = in_grid(i + k / 3 - 1, j + k % 3 - 1, D.n) ? s[k] : 0.f;
}

}  // namespace mg

namespace mg {
// out = P xc
__global__ void k_t_P(TrainDims D, const float* __restrict__ xc, float* __restrict__ out) {
  const int vec = blockIdx.y;
  const int q = blockIdx.x * TT + threadIdx.x;
  if (q >= (int)D.nn) return;
  const int i = q / D.n, j = q % D.n;
  const float* c = xc + (size_t)vec * D.nnc;
  float v = 0.f;
  for (int di = -1; di <= 1; ++di)
    for (int dj = -1; dj <= 1; ++dj) {
      const int fi = i + di, fj = j + dj;
      if ((fi & 1) && (fj & 1)) {
        const int I = (fi - 1) >> 1, J = (fj - 1) >> 1;
        if (in_grid(I, J, D.nc)) v += (di ? 0.5f : 1.f) * (dj ? 0.5f : 1.f) * c[I * D.nc + J];
      }
    }
  out[(size_t)vec * D.nn + q] = v;
}
}  // namespace mg

using namespace mg;

struct mg_train_ctx {
  TrainDims D;
  int bf16 = 0;
  float omega = 2.f / 3.f;
  float* s9 = nullptr;
  float* fields = nullptr;
  float* cfields = nullptr;
  float* W = nullptr;
  float* dW = nullptr;
  ProbDev* probs = nullptr;
  double* band = nullptr;
  double* ut = nullptr;
  double* ybuf = nullptr;
  float *v0 = nullptr, *e1 = nullptr, *e2 = nullptr, *v2 = nullptr, *g3 = nullptr, *t = nullptr, *g2 = nullptr,
        *g1 = nullptr, *rc = nullptr, *xc = nullptr;
  float* loss_partial = nullptr;
  float* param_partial = nullptr;
  int* fail = nullptr;
  int ncta_bw = 0;
  int kmax = 1, k = 1, ckpt = 0;   // cycles reserved / used by the loss; checkpointing
  int arch = MG_NET_CONV;          // network architecture (mg_net_arch)
  float* fc_scratch = nullptr;     // the fully connected network's backward tape
  float* lw[6] = {};               // the linear smoother: w1..w4 and two adjoint vectors;
                                   // the three-kernel stack: lw[0..3]
  float* lpart = nullptr;          // its per-CTA correlation partials
  float* lgrad = nullptr;          // its gradient accumulator [MG_NPARAMS_LIN]
  float* sh_params = nullptr;      // MG_NET_CONV_SHARED: the set in the dense layout
  float* sh_grad = nullptr;        // and the dense gradient
  std::vector<float*> X;           // X[c]: input of cycle c >= 1
  std::vector<float*> V0, V2;      // A e_c and A (C S e_c) of cycle c (V0[0] = v0, V2[0] = v2)
  std::vector<float> h_s9;
  std::vector<ProbDev> h_probs;
};

namespace {

constexpr int kMaxTrainCycles = 16;

mg_status train_dims(const mg_problem* probs, int nprob, int nvec, const mg_options* o, TrainDims& D, int& is_const) {
  if (!probs || nprob < 1 || nvec < 1 || !o) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "training: bad arguments");
  if (o->train_cycles < 0 || o->train_cycles > kMaxTrainCycles)
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "train_cycles must be in [0, %d]", kMaxTrainCycles);
  if (o->net_arch != MG_NET_CONV && o->net_arch != MG_NET_FC && o->net_arch != MG_NET_LINEAR &&
      o->net_arch != MG_NET_CONV_SHARED && o->net_arch != MG_NET_CONV3)
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "unknown net_arch");
  if (o->net_arch == MG_NET_CONV3 && o->conv_bf16)
    return (mg_status)api_fail(MG_ERR_UNSUPPORTED, "the three-kernel network trains in FP32 (conv_bf16 = 0)");
  if ((long long)nprob * nvec > 65535) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "nprob * nvec must be <= 65535");
  if (!(o->omega > 0.f) || !(o->omega < 2.f)) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "omega must be in (0, 2)");
  const int n = probs[0].n;
  if (n != 7 && n != 15 && n != 31 && n != 63)
    return (mg_status)api_fail(MG_ERR_UNSUPPORTED, "training grids must be 7, 15, 31 or 63 (got %d)", n);
  int nconst = 0;
  for (int p = 0; p < nprob; ++p) {
    if (probs[p].n != n) return (mg_status)api_fail(MG_ERR_UNSUPPORTED, "all training problems must share n");
    const int k = probs[p].kind;
    if (k == MG_PROBLEM_ROTATED) {
      if (!(probs[p].eps > 0.0)) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "problem %d: eps must be > 0", p);
      ++nconst;
    } else if (k == MG_PROBLEM_STENCIL) {
      if (!probs[p].data) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "problem %d: NULL stencil", p);
      ++nconst;
    } else if (k == MG_PROBLEM_VARCOEF5 || k == MG_PROBLEM_FIELD) {
      if (!probs[p].data) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "problem %d: NULL data", p);
    } else {
      return (mg_status)api_fail(MG_ERR_INVALID_ARG, "problem %d: unknown kind", p);
    }
  }
  if (nconst != 0 && nconst != nprob)
    return (mg_status)api_fail(MG_ERR_UNSUPPORTED, "a training batch mixes constant and per-point problems");
  is_const = nconst > 0;
  D.n = n;
  D.nc = (n - 1) / 2;
  D.B = nprob;
  D.Z = nvec;
  D.w = D.nc + 1;
  D.nn = (size_t)n * n;
  D.nnc = (size_t)D.nc * D.nc;
  return MG_OK;
}

template <class T>
T* take(char* base, size_t& off, size_t count) {
  off = (off + 255) & ~(size_t)255;
  T* p = base ? (T*)(base + off) : nullptr;
  off += count * sizeof(T);
  return p;
}

size_t train_carve(const TrainDims& D, int kmax, int ckpt, int arch, void* basev, mg_train_ctx* c) {
  char* base = (char*)basev;
  size_t off = 0;
  const size_t BZ = (size_t)D.B * D.Z, m = D.nnc, ld = D.w + 1;
  mg_train_ctx tmp;
  mg_train_ctx& x = c ? *c : tmp;
  x.s9 = take<float>(base, off, 9 * (size_t)D.B);
  x.fields = take<float>(base, off, 9 * D.nn * D.B);
  x.cfields = take<float>(base, off, 9 * D.nnc * D.B);
  const size_t nk = arch == MG_NET_CONV3 ? 3 : 1;  // kernels per point
  x.W = take<float>(base, off, 9 * nk * D.nn * D.B);
  x.dW = take<float>(base, off, 9 * nk * D.nn * D.B);
  x.probs = take<ProbDev>(base, off, D.B);
  x.band = take<double>(base, off, m * ld * D.B);
  x.ut = take<double>(base, off, m * ld * D.B);
  x.ybuf = take<double>(base, off, m * BZ);
  float** vecs[] = {&x.v0, &x.e1, &x.e2, &x.v2, &x.g3, &x.t, &x.g2, &x.g1};
  for (float** v : vecs) *v = take<float>(base, off, D.nn * BZ);
  x.X.assign(kmax, nullptr);
  x.V0.assign(kmax, x.v0);
  x.V2.assign(kmax, x.v2);
  for (int c = 1; c < kmax; ++c) {
    x.X[c] = take<float>(base, off, D.nn * BZ);
    if (!ckpt) {
      x.V0[c] = take<float>(base, off, D.nn * BZ);
      x.V2[c] = take<float>(base, off, D.nn * BZ);
    }
  }
  x.rc = take<float>(base, off, D.nnc * BZ);
  x.xc = take<float>(base, off, D.nnc * BZ);
  x.loss_partial = take<float>(base, off, BZ);
  x.ncta_bw = net_backward_ctas(D.n, D.B);
  x.param_partial = take<float>(base, off, (size_t)x.ncta_bw * (arch == MG_NET_CONV3 ? MG_NPARAMS_K3 : MG_NPARAMS));
  if (arch == MG_NET_CONV3)  // K1 v, K2 K1 v and two adjoint vectors of the stack
    for (int k = 0; k < 4; ++k) x.lw[k] = take<float>(base, off, D.nn * BZ);
  x.fc_scratch = arch == MG_NET_FC ? take<float>(base, off, fc_backward_floats(D.n, D.B)) : nullptr;
  if (arch == MG_NET_LINEAR) {
    for (int k = 0; k < 6; ++k) x.lw[k] = take<float>(base, off, D.nn * BZ);
    x.lpart = take<float>(base, off, ((D.nn + TT - 1) / TT) * BZ * 9);
    x.lgrad = take<float>(base, off, MG_NPARAMS_LIN);
  }
  if (arch == MG_NET_CONV_SHARED) {
    x.sh_params = take<float>(base, off, MG_NPARAMS);
    x.sh_grad = take<float>(base, off, MG_NPARAMS);
  }
  x.fail = take<int>(base, off, 4);
  return off + 256;
}

}  // namespace

#define TCK(call)                                                                                       \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return (mg_status)api_fail(MG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" {

size_t mg_train_workspace_size(const mg_problem* problems, int nprob, int nvec, const mg_options* opts) {
  TrainDims D;
  int is_const = 0;
  if (train_dims(problems, nprob, nvec, opts, D, is_const) != MG_OK) return 0;
  return train_carve(D, opts->train_cycles > 1 ? opts->train_cycles : 1, opts->train_checkpoint != 0, opts->net_arch,
                     nullptr, nullptr);
}

mg_status mg_train_setup(const mg_problem* problems, int nprob, int nvec, const mg_options* opts, void* workspace,
                         size_t ws_bytes, void* stream, mg_train_ctx** out) {
  if (!out) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  TrainDims D;
  int is_const = 0;
  mg_status st = train_dims(problems, nprob, nvec, opts, D, is_const);
  if (st != MG_OK) return st;
  const int kmax = opts->train_cycles > 1 ? opts->train_cycles : 1, ckpt = opts->train_checkpoint != 0;
  const size_t need = train_carve(D, kmax, ckpt, opts->net_arch, nullptr, nullptr);
  if (!workspace || ws_bytes < need)
    return (mg_status)api_fail(MG_ERR_WORKSPACE, "training workspace needs %zu bytes, got %zu", need, ws_bytes);
  if (((uintptr_t)workspace & 255) != 0) return (mg_status)api_fail(MG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  mg_train_ctx* c = new mg_train_ctx();
  c->D = D;
  c->bf16 = opts->conv_bf16;
  c->omega = opts->omega;
  c->kmax = c->k = kmax;
  c->ckpt = ckpt;
  c->arch = opts->net_arch;
  train_carve(D, kmax, ckpt, opts->net_arch, workspace, c);
  auto run = [&]() -> mg_status {
    const dim3 gp((unsigned)((D.nn + TT - 1) / TT), D.B);
    if (is_const) {
      c->h_s9.resize(9 * (size_t)D.B);
      for (int p = 0; p < D.B; ++p) {
        float* s9 = &c->h_s9[9 * (size_t)p];
        if (problems[p].kind == MG_PROBLEM_ROTATED) {
          if (mg_rotated_stencil(problems[p].eps, problems[p].theta, s9) != MG_OK) return MG_ERR_INVALID_ARG;
        } else {
          for (int k = 0; k < 9; ++k) s9[k] = problems[p].data[k];
        }
      }
      TCK(cudaMemcpyAsync(c->s9, c->h_s9.data(), sizeof(float) * 9 * D.B, cudaMemcpyHostToDevice, s));
      k_t_const_field<<<gp, TT, 0, s>>>(D, c->s9, c->fields);
    } else {
      for (int p = 0; p < D.B; ++p) {
        float* f = c->fields + (size_t)p * 9 * D.nn;
        if (problems[p].kind == MG_PROBLEM_VARCOEF5) TCK(launch_varcoef5(D.n, 1, problems[p].data, 0, f, 0, s));
        else TCK(cudaMemcpyAsync(f, problems[p].data, sizeof(float) * 9 * D.nn, cudaMemcpyDeviceToDevice, s));
      }
    }
    // two-level descriptors to reuse the Galerkin kernel
    c->h_probs.assign(D.B, ProbDev());
    for (int p = 0; p < D.B; ++p) {
      ProbDev& d = c->h_probs[p];
      memset(&d, 0, sizeof(d));
      d.lv[0].n = D.n;
      d.lv[0].st = c->fields + (size_t)p * 9 * D.nn;
      d.lv[1].n = D.nc;
      d.lv[1].st = c->cfields + (size_t)p * 9 * D.nnc;
    }
    TCK(cudaMemcpyAsync(c->probs, c->h_probs.data(), sizeof(ProbDev) * D.B, cudaMemcpyHostToDevice, s));
    TCK(launch_rap_field(c->probs, D.B, 0, D.nc, s));
    TCK(cudaMemsetAsync(c->fail, 0, sizeof(int), s));
    k_t_band_factor<<<D.B, 256, 0, s>>>(D, c->cfields, c->band, c->fail);
    const int m = D.nc * D.nc, ld = D.w + 1;
    k_t_band_finish<<<dim3((m * ld + 255) / 256, D.B), 256, 0, s>>>(D, c->band, c->ut);
    k_t_band_invdiag<<<dim3((m + 255) / 256, D.B), 256, 0, s>>>(D, c->band);
    TCK(cudaGetLastError());
    return MG_OK;
  };
  st = run();
  if (st != MG_OK) {
    delete c;
    return st;
  }
  *out = c;
  return MG_OK;
}

void mg_train_destroy(mg_train_ctx* ctx) { delete ctx; }

mg_status mg_train_set_cycles(mg_train_ctx* ctx, int cycles) {
  if (!ctx || cycles < 1 || cycles > ctx->kmax)
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "cycles must be in [1, train_cycles of the setup]");
  ctx->k = cycles;
  return MG_OK;
}

static mg_status train_step(mg_train_ctx* c, const float* params, const float* z, const CycleArgs* cf,
                            const CycleArgs* ct, float* grad_out, float* loss_out, void* stream) {
  if (!c || !params || !z || !loss_out) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_train_step: bad arguments");
  const TrainDims& D = c->D;
  cudaStream_t s = (cudaStream_t)stream;
  const int BZ = D.B * D.Z;
  const dim3 gv((unsigned)((D.nn + TT - 1) / TT), BZ), gc((unsigned)((D.nnc + TT - 1) / TT), BZ);
  const int solve_blocks = (BZ * 32 + 127) / 128;
  const float inv = 1.f / ((float)D.nn * D.Z * D.B);
  NetBatch nb;
  nb.st = c->fields;
  nb.W = c->W;
  nb.stride = 9 * D.nn;
  nb.n = D.n;
  nb.pad_ = 0;
  const bool lin = c->arch == MG_NET_LINEAR;  // params are the smoother's 54 weights
  const float* net_prm = params;              // the convolutional network in the dense layout
  if (c->arch == MG_NET_CONV_SHARED) {
    TCK(launch_net_expand_shared(params, c->sh_params, 1, s));
    net_prm = c->sh_params;
  }
  const bool k3 = c->arch == MG_NET_CONV3;  // H = K3 K2 K1, c->W holds [27][n][n] per problem
  if (c->arch == MG_NET_FC) TCK(launch_fc_forward_batch(nb, D.B, params, c->omega, c->bf16, s));
  else if (k3) TCK(launch_net_forward3_batch(nb, D.B, params, c->omega, s));
  else if (!lin) TCK(launch_net_forward_batch(nb, D.B, net_prm, c->omega, c->bf16, s));
  const int K = c->k;
  // out = x - H v
  auto xmHv = [&](const float* x, const float* v, float* out) {
    if (k3) {
      k_t3_conv<<<gv, TT, 0, s>>>(D, c->W, 0, nullptr, v, c->lw[0]);
      k_t3_conv<<<gv, TT, 0, s>>>(D, c->W, 1, nullptr, c->lw[0], c->lw[1]);
      k_t3_conv<<<gv, TT, 0, s>>>(D, c->W, 2, x, c->lw[1], out);
      return;
    }
    if (!lin) {
      k_t_xmHv<<<gv, TT, 0, s>>>(D, c->fields, c->W, x, v, out);
      return;
    }
    k_tl_conv<<<gv, TT, 0, s>>>(D, params, v, c->lw[4]);
    k_tl_conv<<<gv, TT, 0, s>>>(D, params + 9, c->lw[4], c->lw[5]);
    k_tl_conv<<<gv, TT, 0, s>>>(D, params + 18, c->lw[5], c->lw[4]);
    k_tl_conv<<<gv, TT, 0, s>>>(D, params + 27, c->lw[4], c->lw[5]);
    k_tl_xmH<<<gv, TT, 0, s>>>(D, params, x, c->lw[5], v, out);
  };
  // the linear smoother's part of the adjoint of e_out = x - H v with output gradient g:
  // grad -= d<g, H v>/dphi, and t = H^T g
  const int nblk = (int)((D.nn + TT - 1) / TT);
  auto corr = [&](const float* g, const float* u, int slot) {
    k_tl_corr<<<dim3(nblk, BZ), TT, 0, s>>>(D, g, u, c->lpart);
    k_tl_reduce<<<9, TT, 0, s>>>(c->lpart, nblk * BZ, c->lgrad, slot);
  };
  auto lin_adjoint = [&](const float* v, const float* g, float* t) {
    float* const* w = c->lw;  // w1..w4 in lw[0..3], adjoint vectors in lw[4], lw[5]
    k_tl_conv<<<gv, TT, 0, s>>>(D, params, v, w[0]);
    for (int k = 1; k < 4; ++k) k_tl_conv<<<gv, TT, 0, s>>>(D, params + 9 * k, w[k - 1], w[k]);
    corr(g, w[3], 4);  // f5 reads w4
    corr(g, v, 5);     // f6 reads v
    const float* lam = g;
    for (int k = 4; k >= 1; --k) {  // lam <- f_{k+1}^T lam: the gradient at w_k
      float* out = c->lw[4 + (k & 1)];
      k_tl_convT<<<gv, TT, 0, s>>>(D, params + 9 * k, lam, out);
      lam = out;
      corr(lam, k >= 2 ? w[k - 2] : v, k - 1);  // f_k reads w_{k-1} (w_0 = v)
    }
    k_tl_HT<<<gv, TT, 0, s>>>(D, params, lam, g, t);
  };
  // the stack's part of the adjoint of e_out = x - K3 K2 K1 v with output gradient g:
  // dW -= g (x) K2 K1 v, (K3^T g) (x) K1 v, (K2^T K3^T g) (x) v; and t = H^T g
  const dim3 gp3(nblk, D.B);
  auto stack_adjoint = [&](const float* v, const float* g, float* t) {
    float* const* w = c->lw;
    k_t3_conv<<<gv, TT, 0, s>>>(D, c->W, 0, nullptr, v, w[0]);
    k_t3_conv<<<gv, TT, 0, s>>>(D, c->W, 1, nullptr, w[0], w[1]);
    k_t3_dW<<<gp3, TT, 0, s>>>(D, g, w[1], c->dW, 2);
    k_t3_convT<<<gv, TT, 0, s>>>(D, c->W, 2, g, w[2]);
    k_t3_dW<<<gp3, TT, 0, s>>>(D, w[2], w[0], c->dW, 1);
    k_t3_convT<<<gv, TT, 0, s>>>(D, c->W, 1, w[2], w[3]);
    k_t3_dW<<<gp3, TT, 0, s>>>(D, w[3], v, c->dW, 0);
    k_t3_convT<<<gv, TT, 0, s>>>(D, c->W, 0, w[3], t);
  };
  // xc = M rc: the exact coarse solve (banded Cholesky), or one V-cycle of the coarse
  // context (cf), whose transpose ct serves the adjoint
  auto coarse_solve = [&](const CycleArgs* ca) -> cudaError_t {
    if (!ca) {
      k_t_band_solve<<<solve_blocks, 128, 0, s>>>(D, c->band, c->ut, c->rc, c->ybuf, c->xc, BZ);
      return cudaGetLastError();
    }
    CycleArgs a = *ca;
    a.stream = s;
    return launch_tail_vec(a, c->rc, c->xc, D.Z);
  };
  cudaError_t ce = cudaSuccess;
  // one cycle e_out = S C S e_in, keeping v0 = A e_in and v2 = A (C S e_in); e_out may be
  // NULL (recomputation of the products only)
  auto cycle = [&](const float* ein, float* v0, float* v2, float* eout) {
    k_t_applyA<<<gv, TT, 0, s>>>(D, c->fields, ein, v0);
    xmHv(ein, v0, c->e1);
    k_t_restrict<<<gc, TT, 0, s>>>(D, c->fields, c->e1, 1, c->rc);
    if (ce == cudaSuccess) ce = coarse_solve(cf);
    k_t_xmP<<<gv, TT, 0, s>>>(D, c->e1, c->xc, c->e2);
    k_t_applyA<<<gv, TT, 0, s>>>(D, c->fields, c->e2, v2);
    if (eout) xmHv(c->e2, v2, eout);
  };
  // forward: e_{c+1} = S C S e_c; the last output goes to g3
  for (int cc = 0; cc < K; ++cc)
    cycle(cc == 0 ? z : c->X[cc], c->V0[cc], c->V2[cc], cc + 1 < K ? c->X[cc + 1] : c->g3);
  k_t_loss<<<BZ, TT, 0, s>>>(D, c->g3, 2.f * inv, c->g3, c->loss_partial);
  k_t_loss_total<<<1, 32, 0, s>>>(c->loss_partial, BZ, inv, loss_out);
  TCK(ce);
  TCK(cudaGetLastError());
  if (!grad_out) return MG_OK;
  // adjoint, cycles in reverse; g3 = dloss/d(output of cycle cc)
  if (lin) TCK(cudaMemsetAsync(c->lgrad, 0, MG_NPARAMS_LIN * sizeof(float), s));
  if (k3) TCK(cudaMemsetAsync(c->dW, 0, 27 * D.nn * D.B * sizeof(float), s));
  for (int cc = K - 1; cc >= 0; --cc) {
    if (c->ckpt && cc + 1 < K) cycle(cc == 0 ? z : c->X[cc], c->V0[cc], c->V2[cc], nullptr);
    if (lin) lin_adjoint(c->V2[cc], c->g3, c->t);
    else if (k3) stack_adjoint(c->V2[cc], c->g3, c->t);
    else k_t_HT<<<gv, TT, 0, s>>>(D, c->fields, c->W, c->g3, c->t);
    k_t_xmAv<<<gv, TT, 0, s>>>(D, c->fields, c->g3, c->t, c->g2);
    k_t_restrict<<<gc, TT, 0, s>>>(D, c->fields, c->g2, 0, c->rc);
    TCK(coarse_solve(ct));
    k_t_P<<<gv, TT, 0, s>>>(D, c->xc, c->t);
    k_t_xmAv<<<gv, TT, 0, s>>>(D, c->fields, c->g2, c->t, c->g1);
    if (lin || k3) {
      if (lin) lin_adjoint(c->V0[cc], c->g1, c->t);
      else stack_adjoint(c->V0[cc], c->g1, c->t);
      if (cc > 0) k_t_xmAv<<<gv, TT, 0, s>>>(D, c->fields, c->g1, c->t, c->g3);
      continue;
    }
    k_t_dW<<<dim3((unsigned)((D.nn + TT - 1) / TT), D.B), TT, 0, s>>>(D, c->g3, c->V2[cc], c->g1, c->V0[cc], c->dW,
                                                                       cc + 1 < K);
    if (cc > 0) {  // dloss/d(input of cycle cc) = S^T g1
      k_t_HT<<<gv, TT, 0, s>>>(D, c->fields, c->W, c->g1, c->t);
      k_t_xmAv<<<gv, TT, 0, s>>>(D, c->fields, c->g1, c->t, c->g3);
    }
  }
  TCK(ce);
  TCK(cudaGetLastError());
  if (lin) {
    TCK(cudaMemcpyAsync(grad_out, c->lgrad, MG_NPARAMS_LIN * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return MG_OK;
  }
  if (c->arch == MG_NET_FC) TCK(launch_fc_backward(nb, D.B, c->dW, params, c->bf16, c->fc_scratch, 1.f, grad_out, s));
  else if (k3) TCK(launch_net_backward3(nb, D.B, c->dW, params, c->param_partial, 1.f, grad_out, s));
  else if (c->arch == MG_NET_CONV_SHARED) {
    TCK(launch_net_backward(nb, D.B, c->dW, net_prm, c->bf16, c->param_partial, 1.f, c->sh_grad, s));
    TCK(launch_net_reduce_shared(c->sh_grad, grad_out, s));
  } else TCK(launch_net_backward(nb, D.B, c->dW, params, c->bf16, c->param_partial, 1.f, grad_out, s));
  return MG_OK;
}

mg_status mg_train_step(mg_train_ctx* c, const float* params, const float* z, float* grad_out, float* loss_out,
                        void* stream) {
  return train_step(c, params, z, nullptr, nullptr, grad_out, loss_out, stream);
}

mg_status mg_train_step_coarse(mg_train_ctx* c, const float* params, const float* z, mg_ctx* coarse, mg_ctx* coarse_t,
                               float* grad_out, float* loss_out, void* stream) {
  if (!c) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_train_step_coarse: ctx is NULL");
  CycleArgs af, at;
  if (!ctx_tail_args(coarse, &af) || !ctx_tail_args(coarse_t, &at))
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "coarse contexts must hold whole hierarchies of side <= 63");
  const TrainDims& D = c->D;
  if (af.n0 != D.nc || at.n0 != D.nc || af.nprob != D.B || at.nprob != D.B || af.L != at.L)
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "coarse contexts must hold the %d coarse operators of side %d", D.B,
                               D.nc);
  return train_step(c, params, z, &af, &at, grad_out, loss_out, stream);
}

mg_status mg_train_get_coarse_field(const mg_train_ctx* c, int prob, float* out, void* stream) {
  if (!c || !out || prob < 0 || prob >= c->D.B)
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_train_get_coarse_field: bad arguments");
  TCK(cudaMemcpyAsync(out, c->cfields + (size_t)prob * 9 * c->D.nnc, sizeof(float) * 9 * c->D.nnc,
                      cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return MG_OK;
}

}  // extern "C"
