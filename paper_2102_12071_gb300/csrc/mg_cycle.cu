// mg_cycle.cu -- the V-cycle of Algorithm 1 on the error equation, for sm_103a.
//
// One solve iteration for a batch of problems (grid.y = problem):
//   k_residual   r = b - A x with x = x_hi + x_lo (float-float, compensated dot product),
//                ||r||^2, convergence test (Sec. 6.1 stopping rule) by the last CTA.
//   k_down(l)    e_l = H r_l (pre-smoothing from zero), s = r_l - A e_l, r_{l+1} = P^T s
//                (Algorithm 1 lines 1-2), levels with n_l > MG_TAIL_N.
//   k_tail       levels with n_l <= MG_TAIL_N in one CTA per problem, down to the FP64
//                coarsest solve and back up (Algorithm 1 lines 3-9).
//   k_up(l)      e_l += P e_{l+1}, e_l += H (r_l - A e_l) (Algorithm 1 lines 8-9); on
//                level 0 the correction goes straight into x (float-float), e_0 is not stored.
// k_tail_solve runs whole solves of small problems (n_0 <= MG_TAIL_N) in one CTA each.
//
// The cycle on the error equation from e = 0 equals Algorithm 1 applied to x because the
// cycle is linear in (x, b); the outer iterate and residual carry ~48 significand bits.
#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_ops.cuh"

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
// Last-CTA completion of a per-problem sum: every CTA stores its partial; the CTA that
// arrives last adds all partials in float-float and returns true in all its threads.
__device__ bool block_partial_and_last(float v, float* partials, unsigned int* counter, int ntiles,
                                       int tile, float& tot_hi, float& tot_lo) {
  __shared__ float wsum[NT / 32];
  __shared__ bool last;
  __shared__ float fhi[NT / 32], flo[NT / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wsum[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int k = 0; k < NT / 32; ++k) s += wsum[k];
    partials[tile] = s;
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == (unsigned)ntiles - 1u);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  float hi = 0.f, lo = 0.f;
  for (int t = threadIdx.x; t < ntiles; t += NT) ff_add(hi, lo, __ldcg(partials + t), 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o), olo = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, ohi, olo);
  }
  if (lane == 0) { fhi[w] = hi; flo[w] = lo; }
  __syncthreads();
  hi = 0.f; lo = 0.f;
  for (int k = 0; k < NT / 32; ++k) ff_add(hi, lo, fhi[k], flo[k]);
  tot_hi = hi;
  tot_lo = lo;
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

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
  if (block_partial_and_last(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, hi, lo)) {
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

// Convergence decision after residual evaluation number k (= cycles applied so far).
__device__ void decide(ProbState& st, float rr_hi, float rr_lo, float rtol, int max_cycles) {
  const int k = st.iter;
  const float rr = rr_hi + rr_lo, bb = st.bb_hi + st.bb_lo;
  const float rel = sqrtf(rr / bb);
  st.rel = rel;
  st.hist[k % MG_HRING] = rel;
  st.cycles = k;
  st.iter = k + 1;
  if (!isfinite(rel)) { st.status = 3; st.active = 0; }
  else if (rel < rtol) { st.status = 1; st.active = 0; }
  else if (k >= max_cycles) { st.status = 2; st.active = 0; }
}

// ------------------------------------------------------------- k_residual
// r = b - A (x_hi + x_lo), compensated: each product a*x_hi is split exactly with an FMA
// and the running sum is kept as an unevaluated pair (Dot2 of Ogita, Rump & Oishi 2005).
template <int SK>
__global__ void __launch_bounds__(NT) k_residual(const ProbDev* __restrict__ probs, ProbState* __restrict__ state,
                                                 float* __restrict__ partials, int ntiles_max,
                                                 const float* __restrict__ b, const float* __restrict__ xhi,
                                                 const float* __restrict__ xlo, float rtol, int max_cycles) {
  const int p = blockIdx.y;
  if (!state[p].active) return;
  const LevelDev L = probs[p].lv[0];
  const int n = L.n;
  const size_t nn = (size_t)n * n;
  const int ntx = (n + TB - 1) / TB, ntiles = ntx * ntx;
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  constexpr int TS = TB + 2;
  __shared__ float XH[TS * TS], XL[TS * TS];
  const float* xh = xhi + p * nn;
  const float* xl = xlo ? xlo + p * nn : nullptr;
  for (int t = threadIdx.x; t < TS * TS; t += NT) {
    const int i = R0 - 1 + t / TS, j = C0 - 1 + t % TS;
    float h = 0.f, l = 0.f;
    if (in_grid(i, j, n)) {
      h = xh[(size_t)i * n + j];
      if (xl) l = xl[(size_t)i * n + j];
    }
    XH[t] = h;
    XL[t] = l;
  }
  float s[9];
  load_stencil<SK>(L, s);
  __syncthreads();
  const float* bp = b + p * nn;
  float acc = 0.f;
  const int tx = threadIdx.x & 31;
  for (int ty = threadIdx.x >> 5; ty < TB; ty += NT / 32) {
    const int i = R0 + ty, j = C0 + tx;
    if (!in_grid(i, j, n)) continue;
    const int c = (ty + 1) * TS + tx + 1;
    float hi = bp[(size_t)i * n + j], lo = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int off = (k / 3 - 1) * TS + (k % 3 - 1);
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
    L.r[(size_t)i * n + j] = r;
    acc = fmaf(r, r, acc);
  }
  float rhi, rlo;
  if (block_partial_and_last(acc, partials + (size_t)p * ntiles_max, &state[p].counter, ntiles, tile, rhi, rlo)) {
    if (threadIdx.x == 0) decide(state[p], rhi, rlo, rtol, max_cycles);
  }
}

// ----------------------------------------------------------------- k_down
template <int SK, int HK>
__global__ void __launch_bounds__(NT) k_down(const ProbDev* __restrict__ probs, const ProbState* __restrict__ state,
                                             int l, float omega) {
  const int p = blockIdx.y;
  if (!state[p].active) return;
  const LevelDev L = probs[p].lv[l];
  const LevelDev Lc = probs[p].lv[l + 1];
  const int n = L.n, nc = Lc.n;
  const int ntx = (n + TB - 1) / TB;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  constexpr int RS = TB + 5, ES = TB + 3, SS = TB + 1;  // r rows R0-2.., e rows R0-1.., s rows R0..
  __shared__ float rs[RS * RS], es[ES * ES], ss[SS * SS];
  __shared__ float wtab[9 * MG_PROXY * MG_PROXY];
  float s[9];
  load_stencil<SK>(L, s);
  if (HK == HK_TABLE) {
    const int cnt = 9 * L.T * L.T;
    for (int t = threadIdx.x; t < cnt; t += NT) wtab[t] = L.W[t];
  }
  for (int t = threadIdx.x; t < RS * RS; t += NT) {
    const int i = R0 - 2 + t / RS, j = C0 - 2 + t % RS;
    rs[t] = in_grid(i, j, n) ? L.r[(size_t)i * n + j] : 0.f;
  }
  __syncthreads();
  // pre-smoothing from zero: e = H r on rows/cols [R0-1, R0+TB+1]
  for (int t = threadIdx.x; t < ES * ES; t += NT) {
    const int ti = t / ES, tj = t % ES;
    const int i = R0 - 1 + ti, j = C0 - 1 + tj;
    float v = 0.f;
    if (in_grid(i, j, n)) {
      v = smoother_apply<SK, HK>(L, s, wtab, omega, i, j, rs + (ti + 1) * RS + tj + 1, RS);
      if (ti >= 1 && ti <= TB && tj >= 1 && tj <= TB) L.e[(size_t)i * n + j] = v;
    }
    es[t] = v;
  }
  __syncthreads();
  // s = r - A e on rows/cols [R0, R0+TB]
  for (int t = threadIdx.x; t < SS * SS; t += NT) {
    const int ti = t / SS, tj = t % SS;
    const int i = R0 + ti, j = C0 + tj;
    float v = 0.f;
    if (in_grid(i, j, n))
      v = rs[(ti + 2) * RS + tj + 2] - stencil_apply<SK>(L, s, i, j, es + (ti + 1) * ES + tj + 1, ES);
    ss[t] = v;
  }
  __syncthreads();
  // r_c = P^T s for the TB/2 x TB/2 coarse points whose centre 2I+1 lies in the tile
  for (int t = threadIdx.x; t < (TB / 2) * (TB / 2); t += NT) {
    const int I = R0 / 2 + t / (TB / 2), J = C0 / 2 + t % (TB / 2);
    if (I < nc && J < nc) {
      const int ci = 2 * I + 1 - R0, cj = 2 * J + 1 - C0;  // 1 .. TB-1
      Lc.r[(size_t)I * nc + J] = restrict_at(ss + ci * SS + cj, SS);
    }
  }
}

// ------------------------------------------------------------------- k_up
// UPDX: level 0, add the final correction to the float-float iterate instead of storing it.
template <int SK, int HK, bool UPDX>
__global__ void __launch_bounds__(NT) k_up(const ProbDev* __restrict__ probs, const ProbState* __restrict__ state,
                                           int l, float omega, float* __restrict__ xhi, float* __restrict__ xlo) {
  const int p = blockIdx.y;
  if (!state[p].active) return;
  const LevelDev L = probs[p].lv[l];
  const LevelDev Lc = probs[p].lv[l + 1];
  const int n = L.n, nc = Lc.n;
  const int ntx = (n + TB - 1) / TB;
  const int tile = blockIdx.x;
  if (tile >= ntx * ntx) return;
  const int R0 = (tile / ntx) * TB, C0 = (tile % ntx) * TB;
  constexpr int CS = TB / 2 + 3;   // coarse rows R0/2-2 .. R0/2+TB/2
  constexpr int E1S = TB + 4;      // fine rows R0-2 .. R0+TB+1
  constexpr int TS = TB + 2;       // fine rows R0-1 .. R0+TB
  __shared__ float ecs[CS * CS], e1s[E1S * E1S], ts[TS * TS];
  __shared__ float wtab[9 * MG_PROXY * MG_PROXY];
  float s[9];
  load_stencil<SK>(L, s);
  if (HK == HK_TABLE) {
    const int cnt = 9 * L.T * L.T;
    for (int t = threadIdx.x; t < cnt; t += NT) wtab[t] = L.W[t];
  }
  const int I0 = R0 / 2 - 2, J0 = C0 / 2 - 2;
  for (int t = threadIdx.x; t < CS * CS; t += NT) {
    const int I = I0 + t / CS, J = J0 + t % CS;
    ecs[t] = in_grid(I, J, nc) ? Lc.e[(size_t)I * nc + J] : 0.f;
  }
  __syncthreads();
  // e1 = e + P e_c on fine rows/cols [R0-2, R0+TB+1]
  for (int t = threadIdx.x; t < E1S * E1S; t += NT) {
    const int i = R0 - 2 + t / E1S, j = C0 - 2 + t % E1S;
    float v = 0.f;
    if (in_grid(i, j, n)) v = L.e[(size_t)i * n + j] + prolong_at(i, j, ecs, I0, J0, CS);
    e1s[t] = v;
  }
  __syncthreads();
  // t = r - A e1 on rows/cols [R0-1, R0+TB]
  for (int t = threadIdx.x; t < TS * TS; t += NT) {
    const int ti = t / TS, tj = t % TS;
    const int i = R0 - 1 + ti, j = C0 - 1 + tj;
    float v = 0.f;
    if (in_grid(i, j, n))
      v = L.r[(size_t)i * n + j] - stencil_apply<SK>(L, s, i, j, e1s + (ti + 1) * E1S + tj + 1, E1S);
    ts[t] = v;
  }
  __syncthreads();
  // post-smoothing: e = e1 + H t on the owned TB x TB points
  const size_t nn = (size_t)n * n;
  const int tx = threadIdx.x & 31;
  for (int ty = threadIdx.x >> 5; ty < TB; ty += NT / 32) {
    const int i = R0 + ty, j = C0 + tx;
    if (!in_grid(i, j, n)) continue;
    const float e = e1s[(ty + 2) * E1S + tx + 2] +
                    smoother_apply<SK, HK>(L, s, wtab, omega, i, j, ts + (ty + 1) * TS + tx + 1, TS);
    const size_t g = (size_t)i * n + j;
    if (UPDX) {
      float* xh = xhi + p * nn;
      if (xlo) {
        float* xl = xlo + p * nn;
        float hi = xh[g], lo = xl[g], sum, err;
        two_sum(hi, e, sum, err);
        err += lo;
        fast_two_sum(sum, err, hi, lo);
        xh[g] = hi;
        xl[g] = lo;
      } else {
        xh[g] += e;
      }
    } else {
      L.e[g] = e;
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
template <int SK, int HK>
__device__ void tail_cycle(const ProbDev& P, float* sm, const TailLayout& lay, const float (*sc)[9], int l0,
                           int L, float omega) {
  const int nt = blockDim.x;
  for (int l = l0; l < L - 1; ++l) {
    const LevelDev& Lv = P.lv[l];
    const int n = Lv.n, nc = P.lv[l + 1].n;
    float* r = sm + lay.off_r[l];
    float* e = sm + lay.off_e[l];
    float* t = sm + lay.off_t;
    const float* w = sm + lay.off_w[l];
    for (int q = threadIdx.x; q < n * n; q += nt) e[q] = tail_H<SK, HK>(Lv, sc[l], w, omega, r, n, q / n, q % n);
    __syncthreads();
    for (int q = threadIdx.x; q < n * n; q += nt) t[q] = r[q] - tail_A<SK>(Lv, sc[l], e, n, q / n, q % n);
    __syncthreads();
    float* rc = sm + lay.off_r[l + 1];
    for (int q = threadIdx.x; q < nc * nc; q += nt) {
      const int I = q / nc, J = q % nc;
      rc[q] = restrict_at(t + (2 * I + 1) * n + 2 * J + 1, n);
    }
    __syncthreads();
  }
  // coarsest: FP64 Cholesky solve, e_L = A_L^{-1} r_L
  {
    const float* r = sm + lay.off_r[L - 1];
    float* e = sm + lay.off_e[L - 1];
    const int m = P.m;
    if (threadIdx.x == 0) {
      double y[64];
      const double* C = P.chol;
      for (int i = 0; i < m; ++i) {
        double v = (double)r[i];
        for (int k = 0; k < i; ++k) v -= C[i * m + k] * y[k];
        y[i] = v / C[i * m + i];
      }
      for (int i = m - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < m; ++k) v -= C[k * m + i] * y[k];
        y[i] = v / C[i * m + i];
      }
      for (int i = 0; i < m; ++i) e[i] = (float)y[i];
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
    for (int q = threadIdx.x; q < n * n; q += nt) {
      const int i = q / n, j = q % n;
      float v = 0.f;
      for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
          const int fi = i + di, fj = j + dj;  // candidate coarse centre 2I+1
          if ((fi & 1) && (fj & 1)) {
            const int I = (fi - 1) >> 1, J = (fj - 1) >> 1;
            if (in_grid(I, J, nc)) v += (di ? 0.5f : 1.f) * (dj ? 0.5f : 1.f) * ec[I * nc + J];
          }
        }
      e[q] += v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n * n; q += nt) t[q] = r[q] - tail_A<SK>(Lv, sc[l], e, n, q / n, q % n);
    __syncthreads();
    for (int q = threadIdx.x; q < n * n; q += nt) e[q] += tail_H<SK, HK>(Lv, sc[l], w, omega, t, n, q / n, q % n);
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
                                                       float omega) {
  extern __shared__ float sm[];
  __shared__ float sc[MG_MAXL][9];
  const int p = blockIdx.x;
  if (!state[p].active) return;
  const ProbDev& P = probs[p];
  int nl[MG_MAXL];
  for (int l = 0; l < L; ++l) nl[l] = P.lv[l].n;
  TailLayout lay;
  tail_layout(nl, l0, L, HK, lay);
  tail_prologue<SK, HK>(P, sm, lay, sc, l0, L);
  const int n = nl[l0];
  float* r = sm + lay.off_r[l0];
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) r[q] = P.lv[l0].r[q];
  __syncthreads();
  tail_cycle<SK, HK>(P, sm, lay, sc, l0, L, omega);
  const float* e = sm + lay.off_e[l0];
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) P.lv[l0].e[q] = e[q];
}

// Whole solves of small problems: up to `budget` iterations of (residual, test, V-cycle,
// update); with `final_residual` one more residual evaluation at the end.
template <int SK, int HK>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_solve(const ProbDev* __restrict__ probs,
                                                             ProbState* __restrict__ state, int L, float omega,
                                                             const float* __restrict__ b, float* __restrict__ xhi,
                                                             float* __restrict__ xlo, float rtol, int max_cycles,
                                                             int budget, int final_residual) {
  extern __shared__ float sm[];
  __shared__ float sc[MG_MAXL][9];
  __shared__ float wh[TAIL_THREADS / 32], wl[TAIL_THREADS / 32];
  __shared__ int go;
  const int p = blockIdx.x;
  if (!state[p].active) return;
  const ProbDev& P = probs[p];
  int nl[MG_MAXL];
  for (int l = 0; l < L; ++l) nl[l] = P.lv[l].n;
  TailLayout lay;
  tail_layout(nl, 0, L, HK, lay);
  tail_prologue<SK, HK>(P, sm, lay, sc, 0, L);
  const LevelDev& L0 = P.lv[0];
  const int n = nl[0];
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
#define MG_DISPATCH(SKv, HKv, CALL)                                                       \
  do {                                                                                    \
    if ((SKv) == SK_CONST && (HKv) == HK_JACOBI) { constexpr int SK_ = SK_CONST, HK_ = HK_JACOBI; CALL; } \
    else if ((SKv) == SK_CONST && (HKv) == HK_TABLE) { constexpr int SK_ = SK_CONST, HK_ = HK_TABLE; CALL; } \
    else if ((SKv) == SK_FIELD && (HKv) == HK_JACOBI) { constexpr int SK_ = SK_FIELD, HK_ = HK_JACOBI; CALL; } \
    else { constexpr int SK_ = SK_FIELD, HK_ = HK_FIELD; CALL; }                          \
  } while (0)

int tiles_per_side(int n) { return (n + TB - 1) / TB; }

cudaError_t launch_bnorm(const CycleArgs& a, const float* b) {
  const int nt = tiles_per_side(a.n0);
  dim3 grid(nt * nt, a.nprob);
  a.prof->launches++;
  k_bnorm<<<grid, NT, 0, a.stream>>>(a.probs, a.state, a.partials, a.ntiles_max, b);
  return cudaGetLastError();
}

cudaError_t launch_residual(const CycleArgs& a, const float* b, const float* xhi, const float* xlo, float rtol,
                            int max_cycles) {
  const int nt = tiles_per_side(a.n0);
  dim3 grid(nt * nt, a.nprob);
  a.prof->launches++;
  a.prof->begin(PK_RESIDUAL, a.stream);
  if (a.sk == SK_CONST)
    k_residual<SK_CONST><<<grid, NT, 0, a.stream>>>(a.probs, a.state, a.partials, a.ntiles_max, b, xhi, xlo, rtol, max_cycles);
  else
    k_residual<SK_FIELD><<<grid, NT, 0, a.stream>>>(a.probs, a.state, a.partials, a.ntiles_max, b, xhi, xlo, rtol, max_cycles);
  a.prof->end(a.stream);
  return cudaGetLastError();
}

size_t tail_smem_bytes(const int* nl, int l0, int L, int hk) {
  TailLayout lay;
  tail_layout(nl, l0, L, hk, lay);
  return (size_t)lay.total * sizeof(float);
}

template <int SK, int HK>
static cudaError_t set_tail_attrs(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_tail<SK, HK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tail_solve<SK, HK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_cycle(const CycleArgs& a, float* xhi, float* xlo) {
  const int L = a.L, ls = a.lstar;
  for (int l = 0; l < ls; ++l) {
    const int nt = tiles_per_side(a.nl[l]);
    dim3 grid(nt * nt, a.nprob);
    a.prof->launches++;
    a.prof->begin(l == 0 ? PK_DOWN0 : PK_DOWN, a.stream);
    MG_DISPATCH(a.sk, a.hk, (k_down<SK_, HK_><<<grid, NT, 0, a.stream>>>(a.probs, a.state, l, a.omega)));
    a.prof->end(a.stream);
  }
  {
    const size_t smem = tail_smem_bytes(a.nl, ls, L, a.hk);
    cudaError_t e;
    MG_DISPATCH(a.sk, a.hk, (e = set_tail_attrs<SK_, HK_>(smem)));
    if (e != cudaSuccess) return e;
    a.prof->launches++;
    a.prof->begin(PK_TAIL, a.stream);
    MG_DISPATCH(a.sk, a.hk, (k_tail<SK_, HK_><<<a.nprob, TAIL_THREADS, smem, a.stream>>>(a.probs, a.state, ls, L, a.omega)));
    a.prof->end(a.stream);
  }
  for (int l = ls - 1; l >= 0; --l) {
    const int nt = tiles_per_side(a.nl[l]);
    dim3 grid(nt * nt, a.nprob);
    a.prof->launches++;
    a.prof->begin(l == 0 ? PK_UP0 : PK_UP, a.stream);
    if (l == 0)
      MG_DISPATCH(a.sk, a.hk, (k_up<SK_, HK_, true><<<grid, NT, 0, a.stream>>>(a.probs, a.state, l, a.omega, xhi, xlo)));
    else
      MG_DISPATCH(a.sk, a.hk, (k_up<SK_, HK_, false><<<grid, NT, 0, a.stream>>>(a.probs, a.state, l, a.omega, nullptr, nullptr)));
    a.prof->end(a.stream);
  }
  return cudaGetLastError();
}

cudaError_t launch_tail_solve(const CycleArgs& a, const float* b, float* xhi, float* xlo, float rtol, int max_cycles,
                              int budget, int final_residual) {
  const size_t smem = tail_smem_bytes(a.nl, 0, a.L, a.hk);
  cudaError_t e;
  MG_DISPATCH(a.sk, a.hk, (e = set_tail_attrs<SK_, HK_>(smem)));
  if (e != cudaSuccess) return e;
  a.prof->launches++;
  a.prof->begin(PK_TAIL, a.stream);
  MG_DISPATCH(a.sk, a.hk, (k_tail_solve<SK_, HK_><<<a.nprob, TAIL_THREADS, smem, a.stream>>>(
                              a.probs, a.state, a.L, a.omega, b, xhi, xlo, rtol, max_cycles, budget, final_residual)));
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
