// mg_tail.cuh -- coarse levels of the V-cycle held entirely in shared memory: the level
// layout, stencil and smoother taps on ring-padded arrays, and the one-CTA recursion from
// a level down to the FP64 coarsest solve and back (Algorithm 1).
#pragma once
#include "mg_common.cuh"
#include "mg_ops.cuh"
#include "mg_tma.cuh"

namespace mg {

// Levels l0 .. L-1 of one problem in one CTA with every vector in shared memory.  Each
// level vector is stored with a one-point ring of zeros (side n+2), so stencil, smoother
// and transfer taps need no bounds checks: the ring is the Dirichlet exterior.
struct TailLayout {
  int n[MG_MAXL];  // level sides
  int off_r[MG_MAXL], off_e[MG_MAXL], off_t[MG_MAXL], off_w[MG_MAXL];
  int off_inv;     // FP64 inverse of the coarsest operator (8-byte aligned)
  int off_s1, off_s2;  // HK_LINEAR: two ring-padded scratch arrays of the first level's size
  int total;       // floats
};

// class tables and the coarsest inverse after the level vectors starting at float offset o
__host__ __device__ inline void tail_layout_tables(const int* nl, int l0, int L, int hk, int o, TailLayout& t) {
  for (int l = 0; l < L; ++l) t.n[l] = nl[l];
  for (int l = l0; l < L; ++l) {
    t.off_w[l] = o;
    if (hk == HK_TABLE && l < L - 1) {
      const int T = nl[l] < MG_PROXY ? nl[l] : MG_PROXY;
      o += 9 * T * T;
    } else if (hk == HK_LINEAR && l < L - 1) {
      o += MG_NPARAMS_LIN;
    }
  }
  t.off_s1 = t.off_s2 = -1;
  if (hk == HK_LINEAR || hk == HK_STACK3) {
    const int mm = (nl[l0] + 2) * (nl[l0] + 2);
    t.off_s1 = o;
    t.off_s2 = o + mm;
    o += 2 * mm;
  }
  o = (o + 1) & ~1;
  t.off_inv = o;
  const int mm = nl[L - 1] * nl[L - 1];
  o += 2 * mm * mm;
  t.total = o;
}

__host__ __device__ inline void tail_layout(const int* nl, int l0, int L, int hk, TailLayout& t) {
  int o = 0;
  for (int l = l0; l < L; ++l) {
    const int m = nl[l] + 2;
    t.off_r[l] = o; o += m * m;
    t.off_e[l] = o; o += m * m;
    t.off_t[l] = o; o += m * m;
  }
  tail_layout_tables(nl, l0, L, hk, o, t);
}

// sum_t w[t * stride] c[d_t] on a ring-padded array of row stride m, centre tap first
__device__ __forceinline__ float tap9(const float* w, int stride, const float* c, int m) {
  float acc = w[4 * stride] * c[0];
  acc = fmaf(w[0], c[-m - 1], acc);
  acc = fmaf(w[stride], c[-m], acc);
  acc = fmaf(w[2 * stride], c[-m + 1], acc);
  acc = fmaf(w[3 * stride], c[-1], acc);
  acc = fmaf(w[5 * stride], c[1], acc);
  acc = fmaf(w[6 * stride], c[m - 1], acc);
  acc = fmaf(w[7 * stride], c[m], acc);
  acc = fmaf(w[8 * stride], c[m + 1], acc);
  return acc;
}

// A v at (i, j); c points at v(i, j) inside a ring-padded array of row stride m.  Callers
// pass the constant stencil s as a copy in registers.
template <int SK>
__device__ __forceinline__ float pad_A(const LevelDev& L, const float (&s)[9], const float* c, int m, int n, int i,
                                       int j) {
  if (SK == SK_CONST) return tap9(s, 1, c, m);
  const size_t nn = (size_t)n * n;
  const float* a = L.st + (size_t)i * n + j;
  float acc = __ldg(a + 4 * nn) * c[0];
  acc = fmaf(__ldg(a), c[-m - 1], acc);
  acc = fmaf(__ldg(a + nn), c[-m], acc);
  acc = fmaf(__ldg(a + 2 * nn), c[-m + 1], acc);
  acc = fmaf(__ldg(a + 3 * nn), c[-1], acc);
  acc = fmaf(__ldg(a + 5 * nn), c[1], acc);
  acc = fmaf(__ldg(a + 6 * nn), c[m - 1], acc);
  acc = fmaf(__ldg(a + 7 * nn), c[m], acc);
  acc = fmaf(__ldg(a + 8 * nn), c[m + 1], acc);
  return acc;
}

// H v at (i, j) on a ring-padded array; wi holds the interior network kernel of the level
// (a copy in registers: interior points read no weights from memory)
template <int SK, int HK>
__device__ __forceinline__ float pad_H(const LevelDev& L, const float (&s)[9], const float* wtab, const float (&wi)[9],
                                       float omega, const float* c, int m, int n, int i, int j) {
  if (HK == HK_JACOBI) {
    const float d = (SK == SK_CONST) ? s[4] : __ldg(L.st + 4 * (size_t)n * n + (size_t)i * n + j);
    return (omega / d) * c[0];
  }
  if (HK == HK_TABLE) {
    const int T = L.T, M = MG_NET_MARGIN;
    if (T == MG_PROXY && i >= M && i < n - M && j >= M && j < n - M) return tap9(wi, 1, c, m);
    return tap9(wtab + kclass(i, n, T) * T + kclass(j, n, T), T * T, c, m);
  }
  return tap9(L.W + (size_t)i * n + j, n * n, c, m);
}

// interior points of level side n, warp per row and lane per column (no integer division)
#define TAIL_FOR(nside)                          \
  for (int i = warp; i < (nside); i += nwarps) \
    for (int j = lane; j < (nside); j += 32)

// sum_t w[t] c[d_t] on a ring-padded array of row stride m, centre tap first (dot9's order)
__device__ __forceinline__ float conv9(const float* w, const float* c, int m) {
  float acc = w[4] * c[0];
  acc = fmaf(w[0], c[-m - 1], acc);
  acc = fmaf(w[1], c[-m], acc);
  acc = fmaf(w[2], c[-m + 1], acc);
  acc = fmaf(w[3], c[-1], acc);
  acc = fmaf(w[5], c[1], acc);
  acc = fmaf(w[6], c[m - 1], acc);
  acc = fmaf(w[7], c[m], acc);
  acc = fmaf(w[8], c[m + 1], acc);
  return acc;
}

// The shared-kernel linear smoother (Sec. 6, eq. full-coarsening-smoother) on one level of
// side n held ring-padded (stride m = n + 2, zero ring): w_k = f_k(w_{k-1}) for k = 1..4
// from w_0 = u, ping-ponging between s1 and s2 (each pass also writes the zero ring, so the
// scratch serves every level size), then dst (=, or += with acc) f_5(w_4) + f_6(u) on the
// interior.  phi: the level's 54 weights (f_1 .. f_5, f_6).  Barriers between the passes;
// the caller synchronises after the last one.
__device__ inline void tail_linear_H(const float* phi, const float* u, float* dst, bool acc, float* s1, float* s2, int n,
                              int m) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float* src = u;
  for (int k = 0; k < 4; ++k) {
    float* out = (k & 1) ? s2 : s1;
    const float* w = phi + 9 * k;
    for (int i = warp - 1; i <= n; i += nwarps)
      for (int j = lane - 1; j <= n; j += 32) {
        const int q = (i + 1) * m + j + 1;
        out[q] = (i >= 0 && i < n && j >= 0 && j < n) ? conv9(w, src + q, m) : 0.f;
      }
    __syncthreads();
    src = out;
  }
  TAIL_FOR(n) {
    const int q = (i + 1) * m + j + 1;
    const float h = conv9(phi + 36, src + q, m) + conv9(phi + 45, u + q, m);
    dst[q] = acc ? dst[q] + h : h;
  }
}

// The three-kernel stack (MG_NET_CONV3) on one ring-padded level: K1 and K2 into the
// scratch arrays (each pass writes the zero ring), then dst (=, or += with acc) K3 on the
// interior; the per-point kernels come from the level's [27][n][n] field in global memory.
// Barriers between the passes; the caller synchronises after the last one.
__device__ inline void tail_stack_H(const float* W, const float* u, float* dst, bool acc, float* s1, float* s2, int n,
                                   int m) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const size_t nn = (size_t)n * n;
  const float* src = u;
  for (int k = 0; k < 2; ++k) {
    float* out = k ? s2 : s1;
    for (int i = warp - 1; i <= n; i += nwarps)
      for (int j = lane - 1; j <= n; j += 32) {
        const int q = (i + 1) * m + j + 1;
        float v = 0.f;
        if (i >= 0 && i < n && j >= 0 && j < n) {
          float w[9];
#pragma unroll
          for (int t = 0; t < 9; ++t) w[t] = __ldg(W + (size_t)(9 * k + t) * nn + (size_t)i * n + j);
          v = conv9(w, src + q, m);
        }
        out[q] = v;
      }
    __syncthreads();
    src = out;
  }
  TAIL_FOR(n) {
    const int q = (i + 1) * m + j + 1;
    float w[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) w[t] = __ldg(W + (size_t)(18 + t) * nn + (size_t)i * n + j);
    const float h = conv9(w, src + q, m);
    dst[q] = acc ? dst[q] + h : h;
  }
}

// Down and up sweeps from level l0 with r_{l0} already in shared memory; leaves e_{l0}.
// nu1 pre-smoothing steps from e = 0 (the first is e = H r, each further one e += H (r - A e))
// and nu2 post-smoothing steps after the correction (Algorithm 1).  The coarsest level is
// one FP64 product with the precomputed inverse of A_L.
template <int SK, int HK>
__device__ void tail_cycle(const ProbDev& P, float* sm, const TailLayout& lay, const float (*sc)[9],
                           const float (*wi)[9], int l0, int L, float omega) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nu1 = P.nu1 > 1 ? P.nu1 : 1, nu2 = P.nu2 > 1 ? P.nu2 : 1;
  // t = r - A e, then (with smooth) e += H t, on level l; both end with a barrier
  auto residual = [&](int l) {
    const LevelDev& Lv = P.lv[l];
    const int n = lay.n[l], m = n + 2;
    const float* r = sm + lay.off_r[l];
    const float* e = sm + lay.off_e[l];
    float* t = sm + lay.off_t[l];
    float sr[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) sr[k] = sc[l][k];
    TAIL_FOR(n) {
      const int q = (i + 1) * m + j + 1;
      t[q] = r[q] - pad_A<SK>(Lv, sr, e + q, m, n, i, j);
    }
    __syncthreads();
  };
  auto smooth_t = [&](int l) {
    const LevelDev& Lv = P.lv[l];
    const int n = lay.n[l], m = n + 2;
    float* e = sm + lay.off_e[l];
    const float* t = sm + lay.off_t[l];
    const float* w = sm + lay.off_w[l];
    if (HK == HK_LINEAR) {
      tail_linear_H(w, t, e, true, sm + lay.off_s1, sm + lay.off_s2, n, m);
    } else if (HK == HK_STACK3) {
      tail_stack_H(Lv.W, t, e, true, sm + lay.off_s1, sm + lay.off_s2, n, m);
    } else {
      float sr[9], wr[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        sr[k] = sc[l][k];
        wr[k] = wi[l][k];
      }
      TAIL_FOR(n) {
        const int q = (i + 1) * m + j + 1;
        e[q] += pad_H<SK, HK>(Lv, sr, w, wr, omega, t + q, m, n, i, j);
      }
    }
    __syncthreads();
  };
  for (int l = l0; l < L - 1; ++l) {
    const LevelDev& Lv = P.lv[l];
    const int n = lay.n[l], m = n + 2, nc = lay.n[l + 1], mc = nc + 2;
    float* r = sm + lay.off_r[l];
    float* e = sm + lay.off_e[l];
    float* t = sm + lay.off_t[l];
    const float* w = sm + lay.off_w[l];
    if (HK == HK_LINEAR) {
      tail_linear_H(w, r, e, false, sm + lay.off_s1, sm + lay.off_s2, n, m);
    } else if (HK == HK_STACK3) {
      tail_stack_H(Lv.W, r, e, false, sm + lay.off_s1, sm + lay.off_s2, n, m);
    } else {
      float sr[9], wr[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        sr[k] = sc[l][k];
        wr[k] = wi[l][k];
      }
      TAIL_FOR(n) {
        const int q = (i + 1) * m + j + 1;
        e[q] = pad_H<SK, HK>(Lv, sr, w, wr, omega, r + q, m, n, i, j);
      }
    }
    __syncthreads();
    for (int k = 1; k < nu1; ++k) {
      residual(l);
      smooth_t(l);
    }
    residual(l);
    float* rc = sm + lay.off_r[l + 1];
    for (int I = warp; I < nc; I += nwarps)
      for (int J = lane; J < nc; J += 32) rc[(I + 1) * mc + J + 1] = restrict_at(t + (2 * I + 2) * m + 2 * J + 2, m);
    __syncthreads();
  }
  {
    const int nL = lay.n[L - 1], mL = nL + 2, mm = nL * nL;
    const float* r = sm + lay.off_r[L - 1];
    float* e = sm + lay.off_e[L - 1];
    if ((int)threadIdx.x < mm) {
      // row threadIdx.x of the inverse times r, one partial sum per row of r (independent
      // chains; no division in the index arithmetic)
      const double* Ai = reinterpret_cast<const double*>(sm + lay.off_inv) + threadIdx.x * mm;
      double acc0 = 0.0, acc1 = 0.0;
#pragma unroll 4
      for (int a = 0; a < nL; ++a) {
        const float* ra = r + (a + 1) * mL + 1;
        const double* Aa = Ai + a * nL;
        double sa = 0.0;
        for (int b = 0; b < nL; ++b) sa = fma(Aa[b], (double)ra[b], sa);
        if (a & 1) acc1 += sa;
        else acc0 += sa;
      }
      e[(threadIdx.x / nL + 1) * mL + threadIdx.x % nL + 1] = (float)(acc0 + acc1);
    }
    __syncthreads();
  }
  for (int l = L - 2; l >= l0; --l) {
    const int n = lay.n[l], m = n + 2, mc = lay.n[l + 1] + 2;
    float* e = sm + lay.off_e[l];
    const float* ec = sm + lay.off_e[l + 1];
    TAIL_FOR(n) e[(i + 1) * m + j + 1] += prolong_at(i, j, ec, -1, -1, mc);
    __syncthreads();
    for (int k = 0; k < nu2; ++k) {
      residual(l);
      smooth_t(l);
    }
  }
}

// Stencil constants, class tables of levels l0 .. L-2 and the coarsest inverse into shared
// memory by asynchronous copies: every copy of every level is in flight at once (copying
// level by level through registers would wait on each level in turn).  The caller's next
// barrier makes them visible.
template <int SK, int HK>
__device__ void load_level_data(const ProbDev& P, float* sm, const TailLayout& lay, float (*sc)[9], int l0, int L) {
  __shared__ const float* src[MG_MAXL];
  __shared__ int pre[MG_MAXL + 1], dst[MG_MAXL];
  const int nq = L - l0;  // entries: the tables of levels l0 .. L-2, then the inverse
  if ((int)threadIdx.x < nq) {
    const int q = threadIdx.x, l = l0 + q;
    src[q] = q < nq - 1 ? ((HK == HK_TABLE || HK == HK_LINEAR) ? P.lv[l].W : nullptr)
                        : reinterpret_cast<const float*>(P.chol);
    dst[q] = q < nq - 1 ? lay.off_w[l] : lay.off_inv;
  }
  if (SK == SK_CONST && (int)threadIdx.x < 9 * nq) sc[l0 + threadIdx.x / 9][threadIdx.x % 9] = P.lv[l0 + threadIdx.x / 9].s[threadIdx.x % 9];
  if (threadIdx.x == 0) {
    int o = 0;
    for (int q = 0; q < nq; ++q) {
      pre[q] = o;
      const int l = l0 + q;
      if (q < nq - 1) {
        if (HK == HK_TABLE) {
          const int T = lay.n[l] < MG_PROXY ? lay.n[l] : MG_PROXY;
          o += 9 * T * T;
        } else if (HK == HK_LINEAR) {
          o += MG_NPARAMS_LIN;
        }
      } else {
        const int mm = lay.n[L - 1] * lay.n[L - 1];
        o += 2 * mm * mm;
      }
    }
    pre[nq] = o;
  }
  __syncthreads();
  // one 4-byte asynchronous copy per element: every copy of the thread is in flight at once
  // and nothing is staged in registers; the caller's barrier after cp_async_wait_all makes
  // them visible to the CTA
  for (int q = 0; q < nq; ++q) {
    const int cnt = pre[q + 1] - pre[q];
    const float* sq = src[q];
    float* dq = sm + dst[q];
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) cp_async4(dq + k, sq + k);
  }
  cp_async_wait_all();
}

// interior network kernel of each table level, from the shared-memory tables
template <int HK>
__device__ __forceinline__ void load_interior_kernels(const float* sm, const TailLayout& lay, float (*wi)[9], int l0,
                                                      int L) {
  if (HK != HK_TABLE) return;
  const int q = threadIdx.x / 9, k = threadIdx.x % 9, l = l0 + q;
  if (l < L - 1 && lay.n[l] >= MG_PROXY) {
    const int T = MG_PROXY, M = MG_NET_MARGIN;
    wi[l][k] = sm[lay.off_w[l] + k * T * T + M * T + M];
  }
}

// Zero rings, stencil constants, class tables, interior kernels and the coarsest inverse of
// levels l0 .. L-1; ends with a barrier.
template <int SK, int HK>
__device__ void tail_prologue(const ProbDev& P, float* sm, const TailLayout& lay, float (*sc)[9], float (*wi)[9],
                              int l0, int L) {
  load_level_data<SK, HK>(P, sm, lay, sc, l0, L);
  for (int l = l0; l < L; ++l) {
    const int m = lay.n[l] + 2;
    const int offs[3] = {lay.off_r[l], lay.off_e[l], lay.off_t[l]};
    for (int a = 0; a < 3; ++a) {
      float* v = sm + offs[a];
      for (int k = threadIdx.x; k < m; k += blockDim.x) {
        v[k] = 0.f;
        v[(m - 1) * m + k] = 0.f;
        v[k * m] = 0.f;
        v[k * m + m - 1] = 0.f;
      }
    }
  }
  __syncthreads();
  load_interior_kernels<HK>(sm, lay, wi, l0, L);
  __syncthreads();
}

}  // namespace mg
