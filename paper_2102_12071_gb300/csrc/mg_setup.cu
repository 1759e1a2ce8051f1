// mg_setup.cu -- hierarchy set-up kernels: level-0 stencils, Galerkin coarse operators
// P^T A P (Sec. 2.2) under full coarsening with bilinear P (Sec. 6.1), and the FP64
// inverse of the coarsest operator (the direct solve of Algorithm 1).
#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

// -div(a grad u), a constant per cell, edge weight = mean of the two cells sharing the
// edge; unknown (i, j) is mesh node (i+1, j+1) of an (n+1) x (n+1) cell mesh.
__global__ void k_varcoef5_field(int n, const float* __restrict__ cells, float* __restrict__ field,
                                 size_t cells_stride, size_t field_stride) {
  const int p = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const float* a = cells + p * cells_stride;
  float* st = field + p * field_stride;
  const int i = q / n, j = q % n, m = n + 1;
  const size_t nn = (size_t)n * n;
  // edge weights and centre in FP64 (exact for cells within a factor 2^28 of each other),
  // each rounded once to FP32
  const double dE = 0.5 * ((double)a[i * m + j + 1] + (double)a[(i + 1) * m + j + 1]);
  const double dW = 0.5 * ((double)a[i * m + j] + (double)a[(i + 1) * m + j]);
  const double dN = 0.5 * ((double)a[(i + 1) * m + j] + (double)a[(i + 1) * m + j + 1]);
  const double dS = 0.5 * ((double)a[i * m + j] + (double)a[i * m + j + 1]);
  const float wE = (float)dE, wW = (float)dW, wN = (float)dN, wS = (float)dS;
  const float centre = (float)(dE + dW + dN + dS);
  st[0 * nn + q] = 0.f;
  st[1 * nn + q] = i > 0 ? -wS : 0.f;
  st[2 * nn + q] = 0.f;
  st[3 * nn + q] = j > 0 ? -wW : 0.f;
  st[4 * nn + q] = centre;
  st[5 * nn + q] = j + 1 < n ? -wE : 0.f;
  st[6 * nn + q] = 0.f;
  st[7 * nn + q] = i + 1 < n ? -wN : 0.f;
  st[8 * nn + q] = 0.f;
}

// Bilinear weight of fine offset (dy, dx) from a coarse centre (1-D factors 1, 1/2).
__device__ __forceinline__ float pw(int dy, int dx) {
  if (dy < -1 || dy > 1 || dx < -1 || dx > 1) return 0.f;
  return (dy ? 0.5f : 1.f) * (dx ? 0.5f : 1.f);
}

// Galerkin coarse stencil field, one thread per coarse point:
// Ac(I, I+D) = sum_{x near 2I+1} sum_k P(x, I) A(x, x+d_k) P(x+d_k, I+D).
__global__ void k_rap_field(const ProbDev* __restrict__ probs, int l) {
  const int p = blockIdx.y;
  const LevelDev F = probs[p].lv[l], C = probs[p].lv[l + 1];
  const int n = F.n, nc = C.n;
  const int Q = blockIdx.x * blockDim.x + threadIdx.x;
  if (Q >= nc * nc) return;
  const int I = Q / nc, J = Q % nc;
  const size_t nn = (size_t)n * n, nnc = (size_t)nc * nc;
  // products px*py*a are exact (px*py is a power of two), so a float-float sum gives the
  // correctly rounded Galerkin entry
  float acc[9], lo[9];
#pragma unroll
  for (int kc = 0; kc < 9; ++kc) { acc[kc] = 0.f; lo[kc] = 0.f; }
  for (int ai = -1; ai <= 1; ++ai)
    for (int aj = -1; aj <= 1; ++aj) {
      const int xi = 2 * I + 1 + ai, xj = 2 * J + 1 + aj;
      const float px = pw(ai, aj);
      for (int k = 0; k < 9; ++k) {
        const float a = F.st[k * nn + (size_t)xi * n + xj];
        if (a == 0.f) continue;
        const int yi = xi + k / 3 - 1, yj = xj + k % 3 - 1;  // fine neighbour
#pragma unroll
        for (int kc = 0; kc < 9; ++kc) {
          const int ci = I + kc / 3 - 1, cj = J + kc % 3 - 1;
          const float py = pw(yi - (2 * ci + 1), yj - (2 * cj + 1));
          if (py != 0.f) ff_add(acc[kc], lo[kc], px * py * a, 0.f);
        }
      }
    }
#pragma unroll
  for (int kc = 0; kc < 9; ++kc) {
    const int ci = I + kc / 3 - 1, cj = J + kc % 3 - 1;
    C.st[kc * nnc + Q] = in_grid(ci, cj, nc) ? acc[kc] + lo[kc] : 0.f;
  }
}

// Constant stencils: the Galerkin product of a constant stencil with bilinear P is again a
// constant stencil (also at the boundary, where the truncated couplings vanish), so one
// thread per problem computes it level by level on an unbounded grid.
__global__ void k_rap_const(ProbDev* __restrict__ probs, int nprob, int L) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  // The recursion is carried in float-float and only rounded for storage: the weights
  // P(x,I) P(y,J) are powers of two, so every product is exact, and no level inherits the
  // rounding of the level above.  (That matters because bilinear P sums to 4 around a coarse
  // point, so the Galerkin product multiplies a stencil's row sum by 4 per level and would
  // amplify each level's FP32 rounding of the near-zero row sum by 4 per level below it.)
  float sh[9], sl[9];
  for (int k = 0; k < 9; ++k) { sh[k] = probs[p].lv[0].s[k]; sl[k] = 0.f; }
  for (int l = 0; l + 1 < L; ++l) {
    float c[9], lo[9];
    for (int k = 0; k < 9; ++k) { c[k] = 0.f; lo[k] = 0.f; }
    // coarse point at fine origin 0 (coarse centres on even fine indices)
    for (int ai = -1; ai <= 1; ++ai)
      for (int aj = -1; aj <= 1; ++aj) {
        const float px = pw(ai, aj);
        for (int k = 0; k < 9; ++k) {
          const int yi = ai + k / 3 - 1, yj = aj + k % 3 - 1;
          for (int kc = 0; kc < 9; ++kc) {
            const float py = pw(yi - 2 * (kc / 3 - 1), yj - 2 * (kc % 3 - 1));
            if (py != 0.f) {
              ff_add(c[kc], lo[kc], px * py * sh[k], 0.f);
              ff_add(c[kc], lo[kc], px * py * sl[k], 0.f);
            }
          }
        }
      }
    for (int k = 0; k < 9; ++k) {
      sh[k] = c[k];
      sl[k] = lo[k];
      probs[p].lv[l + 1].s[k] = c[k] + lo[k];
    }
  }
}

// Dense FP64 inverse of the coarsest operator (m = n_L^2 <= 64), one thread per problem; the
// coarsest solve of Algorithm 1 is then one FP64 matrix-vector product.
__global__ void k_coarsest_factor(ProbDev* __restrict__ probs, int nprob, int L, int sk, int* __restrict__ fail) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const LevelDev C = probs[p].lv[L - 1];
  const int n = C.n, m = n * n;
  double* A = probs[p].chol;
  for (int q = 0; q < m * m; ++q) A[q] = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < 9; ++k) {
        const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
        if (!in_grid(ii, jj, n)) continue;
        const float a = sk == SK_CONST ? C.s[k] : C.st[(size_t)k * m + i * n + j];
        A[(i * n + j) * m + ii * n + jj] += (double)a;
      }
  // in-place Gauss-Jordan inversion; all pivots of an SPD matrix are positive
  for (int k = 0; k < m; ++k) {
    const double piv = A[k * m + k];
    if (!(piv > 0.0)) {
      atomicExch(fail, 1);
      return;
    }
    A[k * m + k] = 1.0;
    for (int j = 0; j < m; ++j) A[k * m + j] /= piv;
    for (int i = 0; i < m; ++i) {
      if (i == k) continue;
      const double f = A[i * m + k];
      A[i * m + k] = 0.0;
      for (int j = 0; j < m; ++j) A[i * m + j] -= f * A[k * m + j];
    }
  }
}

// Stencil field of (p, l) expanded to [9][n][n] (couplings across the boundary zero).
__global__ void k_expand_stencil(const ProbDev* __restrict__ probs, int p, int l, int sk, float* __restrict__ out) {
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int i = q / n, j = q % n;
  const size_t nn = (size_t)n * n;
  for (int k = 0; k < 9; ++k) {
    float v;
    if (sk == SK_CONST) v = in_grid(i + k / 3 - 1, j + k % 3 - 1, n) ? L.s[k] : 0.f;
    else v = L.st[k * nn + q];
    out[k * nn + q] = v;
  }
}

// Smoothing kernels of (p, l) expanded to one 3x3 kernel per point.
__global__ void k_expand_kernels(const ProbDev* __restrict__ probs, int p, int l, int sk, int hk, float omega,
                                 float* __restrict__ out) {
  const LevelDev L = probs[p].lv[l];
  const int n = L.n;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int i = q / n, j = q % n;
  const size_t nn = (size_t)n * n;
  for (int k = 0; k < 9; ++k) {
    float v = 0.f;
    if (hk == HK_JACOBI) {
      const float d = sk == SK_CONST ? L.s[4] : L.st[4 * nn + q];
      v = k == 4 ? omega / d : 0.f;
    } else if (hk == HK_TABLE) {
      const int T = L.T;
      v = L.W[k * T * T + kclass(i, n, T) * T + kclass(j, n, T)];
    } else {
      v = L.W[k * nn + q];
    }
    out[k * nn + q] = v;
  }
}

cudaError_t launch_varcoef5(int n, int nprob, const float* cells, size_t cells_stride, float* field,
                            size_t field_stride, cudaStream_t s) {
  dim3 grid((n * n + 255) / 256, nprob);
  k_varcoef5_field<<<grid, 256, 0, s>>>(n, cells, field, cells_stride, field_stride);
  return cudaGetLastError();
}

cudaError_t launch_rap_field(ProbDev* probs, int nprob, int l, int nc, cudaStream_t s) {
  dim3 grid((nc * nc + 127) / 128, nprob);
  k_rap_field<<<grid, 128, 0, s>>>(probs, l);
  return cudaGetLastError();
}

cudaError_t launch_rap_const(ProbDev* probs, int nprob, int L, cudaStream_t s) {
  k_rap_const<<<(nprob + 63) / 64, 64, 0, s>>>(probs, nprob, L);
  return cudaGetLastError();
}

cudaError_t launch_coarsest_factor(ProbDev* probs, int nprob, int L, int sk, int* fail, cudaStream_t s) {
  k_coarsest_factor<<<(nprob + 63) / 64, 64, 0, s>>>(probs, nprob, L, sk, fail);
  return cudaGetLastError();
}

cudaError_t launch_expand_stencil(const ProbDev* probs, int p, int l, int n, int sk, float* out, cudaStream_t s) {
  k_expand_stencil<<<(n * n + 255) / 256, 256, 0, s>>>(probs, p, l, sk, out);
  return cudaGetLastError();
}

cudaError_t launch_expand_kernels(const ProbDev* probs, int p, int l, int n, int sk, int hk, float omega, float* out,
                                  cudaStream_t s) {
  k_expand_kernels<<<(n * n + 255) / 256, 256, 0, s>>>(probs, p, l, sk, hk, omega, out);
  return cudaGetLastError();
}

}  // namespace mg
