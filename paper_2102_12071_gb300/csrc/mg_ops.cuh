// mg_ops.cuh -- grid transfers on shared-memory tiles: bilinear prolongation P and its
// transpose, the restriction P^T (Sec. 6.1).
#pragma once
#include "mg_common.cuh"

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
