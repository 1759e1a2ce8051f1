// mg_ops.cuh -- stencil (A) and smoother (H) evaluation on shared-memory tiles.
//
// Tap k = 3*(di+1) + (dj+1) couples point (i, j) to (i+di, j+dj).  Tiles are zero
// outside the grid (homogeneous Dirichlet), so a constant stencil can be applied with
// all nine taps at boundary points.
#pragma once
#include "mg_common.cuh"

// A v at grid point (i, j); c points at v(i, j) inside a tile of row stride ts.
template <int SK>
__device__ __forceinline__ float stencil_apply(const LevelDev& L, const float (&s)[9], int i, int j,
                                               const float* c, int ts) {
  if (SK == SK_CONST) {
    float acc = s[4] * c[0];
    acc = fmaf(s[0], c[-ts - 1], acc);
    acc = fmaf(s[1], c[-ts], acc);
    acc = fmaf(s[2], c[-ts + 1], acc);
    acc = fmaf(s[3], c[-1], acc);
    acc = fmaf(s[5], c[1], acc);
    acc = fmaf(s[6], c[ts - 1], acc);
    acc = fmaf(s[7], c[ts], acc);
    acc = fmaf(s[8], c[ts + 1], acc);
    return acc;
  } else {
    const int n = L.n;
    const size_t nn = (size_t)n * n;
    const float* a = L.st + (size_t)i * n + j;
    float acc = __ldg(a + 4 * nn) * c[0];
    acc = fmaf(__ldg(a), c[-ts - 1], acc);
    acc = fmaf(__ldg(a + nn), c[-ts], acc);
    acc = fmaf(__ldg(a + 2 * nn), c[-ts + 1], acc);
    acc = fmaf(__ldg(a + 3 * nn), c[-1], acc);
    acc = fmaf(__ldg(a + 5 * nn), c[1], acc);
    acc = fmaf(__ldg(a + 6 * nn), c[ts - 1], acc);
    acc = fmaf(__ldg(a + 7 * nn), c[ts], acc);
    acc = fmaf(__ldg(a + 8 * nn), c[ts + 1], acc);
    return acc;
  }
}

// Diagonal of A at (i, j).
template <int SK>
__device__ __forceinline__ float stencil_diag(const LevelDev& L, const float (&s)[9], int i, int j) {
  if (SK == SK_CONST) return s[4];
  return __ldg(L.st + 4 * (size_t)L.n * L.n + (size_t)i * L.n + j);
}

// H v at grid point (i, j).  wtab: class table of this level in shared memory (HK_TABLE).
template <int SK, int HK>
__device__ __forceinline__ float smoother_apply(const LevelDev& L, const float (&s)[9], const float* wtab,
                                                float omega, int i, int j, const float* c, int ts) {
  if (HK == HK_JACOBI) {
    return omega * c[0] / stencil_diag<SK>(L, s, i, j);
  } else {
    const float* w;
    size_t stride;
    if (HK == HK_TABLE) {
      const int T = L.T;
      w = wtab + kclass(i, L.n, T) * T + kclass(j, L.n, T);
      stride = (size_t)T * T;
    } else {
      w = L.W + (size_t)i * L.n + j;
      stride = (size_t)L.n * L.n;
    }
    float acc = w[4 * stride] * c[0];
    acc = fmaf(w[0], c[-ts - 1], acc);
    acc = fmaf(w[stride], c[-ts], acc);
    acc = fmaf(w[2 * stride], c[-ts + 1], acc);
    acc = fmaf(w[3 * stride], c[-1], acc);
    acc = fmaf(w[5 * stride], c[1], acc);
    acc = fmaf(w[6 * stride], c[ts - 1], acc);
    acc = fmaf(w[7 * stride], c[ts], acc);
    acc = fmaf(w[8 * stride], c[ts + 1], acc);
    return acc;
  }
}

// Bilinear interpolation P e_c at fine point (i, j) (Sec. 6.1): coarse point I sits at
// fine 2I+1.  ec(I, J) read through a tile with origin (I0, J0) and row stride ts, zero
// outside the coarse grid.
__device__ __forceinline__ float prolong_at(int i, int j, const float* ec, int I0, int J0, int ts) {
  float v;
  const int Ia = (i - 1) >> 1, Ja = (j - 1) >> 1;  // floor((i-1)/2), i >= 0
  const float* b = ec + (Ia - I0) * ts + (Ja - J0);
  if (i & 1) {
    if (j & 1) v = b[0];
    else v = 0.5f * (b[0] + b[1]);
  } else {
    if (j & 1) v = 0.5f * (b[0] + b[ts]);
    else v = 0.25f * ((b[0] + b[1]) + (b[ts] + b[ts + 1]));
  }
  return v;
}

// P^T s at coarse point (I, J); c points at s(2I+1, 2J+1) in a tile of row stride ts.
__device__ __forceinline__ float restrict_at(const float* c, int ts) {
  const float edge = (c[-ts] + c[ts]) + (c[-1] + c[1]);
  const float corner = (c[-ts - 1] + c[-ts + 1]) + (c[ts - 1] + c[ts + 1]);
  return c[0] + 0.5f * edge + 0.25f * corner;
}
