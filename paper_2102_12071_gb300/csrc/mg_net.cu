// mg_net.cu -- stencil-to-smoother network (Sec. 4.2, Fig. conv; layer sizes of Sec. 6.2).
//
// Per point the input has 9 channels, the point's stencil divided by its diagonal (zero
// outside the grid).  Three 3x3 convolutions 9->7->5->3 with LeakyReLU(0.01), zero padding
// at every layer, then a layer from the 3x3 window of the 3-channel map (27 inputs) to the
// 9 taps of the point's smoothing kernel: W = (omega*delta_4 + out) / diag.
//
// One CTA computes a 16 x 16 tile of outputs; it recomputes the 4-point halo of the three
// convolution layers (receptive field radius 4) so tiles are independent.  With bf16 the
// weights and every layer input are rounded to bfloat16 and products accumulate in FP32.
// The channel counts (<= 9) are far too small for the tensor cores to pay off, so the
// contraction runs on the FP32 pipes; the whole network is ~2.5 kflop per point.
#include <cuda_bf16.h>

#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

constexpr int OT = 16;               // output tile side
constexpr int S0 = OT + 8, S1 = OT + 6, S2 = OT + 4, S3 = OT + 2;
constexpr int NET_THREADS = 256;
constexpr int OFF_W1 = 0, OFF_W2 = 7 * 9 * 9, OFF_W3 = OFF_W2 + 5 * 7 * 9, OFF_WF = OFF_W3 + 3 * 5 * 9;

__device__ __forceinline__ float rnd_bf16(float v, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}
__device__ __forceinline__ float lrelu(float z) { return z > 0.f ? z : 0.01f * z; }

// Stencil tap k at (i, j) of a network job: a field, or a constant stencil on a grid of
// side n whose couplings across the boundary are dropped.
__device__ __forceinline__ float job_tap(const NetJob& J, int k, int i, int j) {
  if (J.st) return J.st[(size_t)k * J.n * J.n + (size_t)i * J.n + j];
  return in_grid(i + k / 3 - 1, j + k % 3 - 1, J.n) ? J.s[k] : 0.f;
}

// Convolution layer over a tile: out[o][y][x] for positions of side so, inputs of side si
// = so + 2, positions outside the grid forced to zero.
template <int CIN, int COUT>
__device__ __forceinline__ void conv_layer(const float* __restrict__ w, const float* in, int si, float* out, int so,
                                           int gy0, int gx0, int n, int bf16) {
  for (int t = threadIdx.x; t < COUT * so * so; t += NET_THREADS) {
    const int o = t / (so * so), pos = t % (so * so);
    const int y = pos / so, x = pos % so;
    float v = 0.f;
    if (in_grid(gy0 + y, gx0 + x, n)) {
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < CIN; ++c) {
        const float* ip = in + c * si * si + y * si + x;
        const float* wp = w + (o * CIN + c) * 9;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) acc = fmaf(wp[ky * 3 + kx], ip[ky * si + kx], acc);
      }
      v = rnd_bf16(lrelu(acc), bf16);
    }
    out[t] = v;
  }
}

// ------------------------------------------------------------------ forward
// One CTA computes a 24 x 24 tile of outputs (the halo the three convolutions need costs
// 1.78x, 1.56x and 1.36x of the tile on their layers, against 1.41x, 1.27x and 1.13x for
// 32 x 32 tiles; but 24 x 24 tiles hold 69 KB of shared memory, so three CTAs fit on an SM
// instead of two, and the kernel, latency-bound, runs 10 % faster at 4095^2).  Each thread computes a run of P consecutive
// positions of one row for every output channel of a layer, so a weight (read by the whole
// warp at once from shared memory, where each (input channel, tap) keeps its output
// channels contiguous) serves P multiply-adds and an input value COUT of them.  The sums
// run over input channel, then kernel row, then kernel column, as in the backward pass.
constexpr int FT = 24;  // forward output tile side
constexpr int F0 = FT + 8, F1 = FT + 6, F2 = FT + 4, F3 = FT + 2;

__host__ __device__ constexpr int pad4(int v) { return (v + 3) & ~3; }
template <int NK>
struct FwdLayout {
  static constexpr int W1 = 0, W2 = W1 + 9 * 9 * pad4(7), W3 = W2 + 7 * 9 * pad4(5), WF = W3 + 5 * 9 * pad4(3);
  static constexpr int NW = WF + 3 * 9 * pad4(9 * NK);
  static constexpr int A = NW, B = A + 9 * F0 * F0;  // a0 (later a2) and a1 (later a3)
  static constexpr int TOTAL = B + 7 * F1 * F1 + 8;  // floats (the last 8: reads past a row end)
};

// conv weights w[o][c][ky][kx] of the parameter vector to wt[(c * 9 + tap) * pad4(COUT) + o]
template <int CIN, int COUT>
__device__ __forceinline__ void load_wt(const float* __restrict__ params, float* wt, int bf16) {
  constexpr int OP = pad4(COUT);
  for (int t = threadIdx.x; t < CIN * 9 * OP; t += NET_THREADS) {
    const int o = t % OP, ct = t / OP;
    wt[t] = o < COUT ? rnd_bf16(params[o * CIN * 9 + ct], bf16) : 0.f;
  }
}

// Layer of side so from inputs of side si = so + 2: out[o][y][x] for every o, positions
// outside the grid forced to zero; with ACT the LeakyReLU (and bf16 rounding) is applied and
// the result stored, otherwise the raw sums are handed to `sink(y, x, acc)`.
template <int CIN, int COUT, int P>
__device__ __forceinline__ void fwd_sums(const float* wt, const float* in, int si, int so, int y, int x0,
                                         float (&acc)[P][COUT]) {
  constexpr int OP = pad4(COUT);
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[p][o] = 0.f;
  // positions past the end of the row repeat the last one (their results are dropped), so
  // every read stays inside the input plane
  int xs[P];
#pragma unroll
  for (int p = 0; p < P; ++p) xs[p] = min(x0 + p, so - 1);
#pragma unroll 1
  for (int c = 0; c < CIN; ++c) {
    const float* ip = in + c * si * si + y * si;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const float* wp = wt + (c * 9 + ky * 3 + kx) * OP;
        float wv[OP];
#pragma unroll
        for (int q = 0; q < OP; q += 4) {
          const float4 v4 = *reinterpret_cast<const float4*>(wp + q);
          wv[q] = v4.x;
          wv[q + 1] = v4.y;
          wv[q + 2] = v4.z;
          wv[q + 3] = v4.w;
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const float iv = ip[ky * si + xs[p] + kx];
#pragma unroll
          for (int o = 0; o < COUT; ++o) acc[p][o] = fmaf(wv[o], iv, acc[p][o]);
        }
      }
  }
}

// The same sums for four consecutive positions x0 .. x0+3 (x0 a multiple of 4) as two
// pairs in packed FP32 (__ffma2_rn: each lane rounded as fmaf, in the same order): per input
// channel and kernel row the six inputs x0 .. x0+5 are three aligned 64-bit loads, and the
// pairs of the middle kernel column are built from them.  The last run of a row reads up to
// two values past the row's end (their results are dropped; the buffers are padded).
template <int CIN, int COUT>
__device__ __forceinline__ void fwd_sums4(const float* wt, const float* in, int si, int y, int x0,
                                          float2 (&acc)[2][COUT]) {
  constexpr int OP = pad4(COUT);
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[h][o] = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int c = 0; c < CIN; ++c) {
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const float* rp = in + c * si * si + (y + ky) * si + x0;
      const float2 v01 = *reinterpret_cast<const float2*>(rp), v23 = *reinterpret_cast<const float2*>(rp + 2),
                   v45 = *reinterpret_cast<const float2*>(rp + 4);
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const float* wp = wt + (c * 9 + ky * 3 + kx) * OP;
        float wv[OP];
#pragma unroll
        for (int q = 0; q < OP; q += 4) {
          const float4 v4 = *reinterpret_cast<const float4*>(wp + q);
          wv[q] = v4.x;
          wv[q + 1] = v4.y;
          wv[q + 2] = v4.z;
          wv[q + 3] = v4.w;
        }
        const float2 a = kx == 0 ? v01 : (kx == 1 ? make_float2(v01.y, v23.x) : v23);
        const float2 b = kx == 0 ? v23 : (kx == 1 ? make_float2(v23.y, v45.x) : v45);
#pragma unroll
        for (int o = 0; o < COUT; ++o) {
          acc[0][o] = __ffma2_rn(make_float2(wv[o], wv[o]), a, acc[0][o]);
          acc[1][o] = __ffma2_rn(make_float2(wv[o], wv[o]), b, acc[1][o]);
        }
      }
    }
  }
}

template <int CIN, int COUT>
__device__ __forceinline__ void fwd_layer(const float* wt, const float* in, int si, float* out, int so, int gy0,
                                          int gx0, int n, int bf16) {
  constexpr int P = 4;
  const int runs = (so + P - 1) / P;
  for (int t = threadIdx.x; t < so * runs; t += NET_THREADS) {
    const int y = t / runs, x0 = (t % runs) * P;
    float2 acc2[2][COUT];
    fwd_sums4<CIN, COUT>(wt, in, si, y, x0, acc2);
    float acc[P][COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) {
      acc[0][o] = acc2[0][o].x;
      acc[1][o] = acc2[0][o].y;
      acc[2][o] = acc2[1][o].x;
      acc[3][o] = acc2[1][o].y;
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int x = x0 + p;
      if (x < so) {
        const bool g = in_grid(gy0 + y, gx0 + x, n);
#pragma unroll
        for (int o = 0; o < COUT; ++o) out[o * so * so + y * so + x] = g ? rnd_bf16(lrelu(acc[p][o]), bf16) : 0.f;
      }
    }
  }
}

// jobs == nullptr: job y is field y of a uniform batch (batch.st + y * batch.stride, its
// NK kernels at batch.W + y * NK * batch.stride).
// NK output kernels per point: NK = 1 gives W = (omega delta + out) / D; NK = 3 the stack
// K1 = (omega delta + out_1) / D, K2 = delta + out_2, K3 = delta + out_3 ([27][n][n] out).
template <int NK>
__global__ void __launch_bounds__(NET_THREADS, 3) k_net_forward(const NetJob* __restrict__ jobs, NetBatch batch,
                                                                const float* __restrict__ params, float omega,
                                                                int bf16) {
  using Lay = FwdLayout<NK>;
  constexpr int NO = 9 * NK;
  extern __shared__ __align__(16) float fsm[];
  float* wt = fsm;
  float* bufA = fsm + Lay::A;  // a0, later a2
  float* bufB = fsm + Lay::B;  // a1, later a3
  NetJob J;
  if (jobs) {
    J = jobs[blockIdx.y];
  } else {
    J.st = batch.st + blockIdx.y * batch.stride;
    J.s = nullptr;
    J.W = batch.W + (size_t)blockIdx.y * batch.stride * NK;
    J.n = batch.n;
  }
  const int n = J.n;
  const int ntx = (n + FT - 1) / FT;
  if ((int)blockIdx.x >= ntx * ntx) return;
  const int oy = (blockIdx.x / ntx) * FT, ox = (blockIdx.x % ntx) * FT;
  load_wt<9, 7>(params + OFF_W1, wt + Lay::W1, bf16);
  load_wt<7, 5>(params + OFF_W2, wt + Lay::W2, bf16);
  load_wt<5, 3>(params + OFF_W3, wt + Lay::W3, bf16);
  load_wt<3, NO>(params + OFF_WF, wt + Lay::WF, bf16);
  // a0: normalised stencil on rows/cols [oy-4, oy+FT+4)
  for (int t = threadIdx.x; t < F0 * F0; t += NET_THREADS) {
    const int i = oy - 4 + t / F0, j = ox - 4 + t % F0;
    if (in_grid(i, j, n)) {
      const float d = job_tap(J, 4, i, j);
#pragma unroll
      for (int c = 0; c < 9; ++c) bufA[c * F0 * F0 + t] = rnd_bf16(job_tap(J, c, i, j) / d, bf16);
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) bufA[c * F0 * F0 + t] = 0.f;
    }
  }
  __syncthreads();
  fwd_layer<9, 7>(wt + Lay::W1, bufA, F0, bufB, F1, oy - 3, ox - 3, n, bf16);
  __syncthreads();
  fwd_layer<7, 5>(wt + Lay::W2, bufB, F1, bufA, F2, oy - 2, ox - 2, n, bf16);
  __syncthreads();
  fwd_layer<5, 3>(wt + Lay::W3, bufA, F2, bufB, F3, oy - 1, ox - 1, n, bf16);
  __syncthreads();
  // output layer over the 3x3 window of the 3-channel map
  constexpr int PF = NK == 1 ? 4 : 1;
  const size_t nn = (size_t)n * n;
  constexpr int runs = FT / PF;
  for (int t = threadIdx.x; t < FT * runs; t += NET_THREADS) {
    const int y = t / runs, x0 = (t % runs) * PF;
    float acc[PF][NO];
    if constexpr (NK == 1) {
      float2 acc2[2][NO];
      fwd_sums4<3, NO>(wt + Lay::WF, bufB, F3, y, x0, acc2);
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        acc[0][o] = acc2[0][o].x;
        acc[1][o] = acc2[0][o].y;
        acc[2][o] = acc2[1][o].x;
        acc[3][o] = acc2[1][o].y;
      }
    } else {
      fwd_sums<3, NO, PF>(wt + Lay::WF, bufB, F3, FT, y, x0, acc);
    }
    const int i = oy + y;
#pragma unroll
    for (int p = 0; p < PF; ++p) {
      const int j = ox + x0 + p;
      if (!in_grid(i, j, n)) continue;
      const float d = job_tap(J, 4, i, j);
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const float v = o < 9 ? ((o == 4 ? omega : 0.f) + acc[p][o]) / d : (o % 9 == 4 ? 1.f : 0.f) + acc[p][o];
        J.W[o * nn + (size_t)i * n + j] = v;
      }
    }
  }
}

template <int NK>
static cudaError_t fwd_prepare() {
  static int done[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(k_net_forward<NK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(FwdLayout<NK>::TOTAL * sizeof(float)));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_net_forward<NK>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = 1;
  return e;
}

template <int NK>
static cudaError_t fwd_launch(const NetJob* jobs, const NetBatch& batch, int ngrids, int nmax, const float* params,
                              float omega, int bf16, cudaStream_t s) {
  cudaError_t e = fwd_prepare<NK>();
  if (e != cudaSuccess) return e;
  const int ntx = (nmax + FT - 1) / FT;
  k_net_forward<NK><<<dim3(ntx * ntx, ngrids), NET_THREADS, FwdLayout<NK>::TOTAL * sizeof(float), s>>>(
      jobs, batch, params, omega, bf16);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ backward
// Gradient of sum_{k,p} dW[k][p] W[k][p] with respect to the parameters, for a uniform
// batch of fields.  Each CTA recomputes the forward pass of its 16 x 16 output tile (with
// halo) and back-propagates the paths that end in its own outputs; summed over tiles this
// is the full gradient.  Rounding to bfloat16 is passed straight through.  Per-CTA
// parameter gradients go to partials[cta][NP] (deterministic reduction after).  NK = 3:
// the three-kernel network, dW [27][n][n] per field at dWall + y * 3 * batch.stride.
template <int NK>
constexpr int bw_smem_floats() {
  return 2 * (NK == 1 ? MG_NPARAMS : MG_NPARAMS_K3) + 9 * S0 * S0 + 7 * S1 * S1 + 5 * S2 * S2 + 3 * S3 * S3 +
         9 * NK * OT * OT + 3 * S3 * S3 + 5 * S2 * S2 + 7 * S1 * S1;
}

// weight gradient of a conv layer: gw[o][c][ky][kx] = sum_{y,x in so x so} dz[o][y][x] in[c][y+ky][x+kx]
template <int CIN, int COUT>
__device__ __forceinline__ void conv_wgrad(const float* dz, int so, const float* in, int si, float* gw) {
  for (int t = threadIdx.x; t < COUT * CIN * 9; t += NET_THREADS) {
    const int o = t / (CIN * 9), c = (t / 9) % CIN, ky = (t % 9) / 3, kx = t % 3;
    const float* d = dz + o * so * so;
    const float* a = in + c * si * si + ky * si + kx;
    float acc = 0.f;
    for (int y = 0; y < so; ++y)
      for (int x = 0; x < so; ++x) acc = fmaf(d[y * so + x], a[y * si + x], acc);
    gw[t] = acc;
  }
}

// input gradient of a conv layer: din[c][y'] = sum_{o,ky,kx} w[o][c][ky][kx] dz[o][y'-ky], then
// times the activation derivative of the layer below (lrelu'(z) from the sign of its output)
// and the domain mask.
template <int CIN, int COUT>
__device__ __forceinline__ void conv_igrad(const float* w, const float* dz, int so, const float* act, int si,
                                           float* dact, int gy0, int gx0, int n) {
  for (int t = threadIdx.x; t < CIN * si * si; t += NET_THREADS) {
    const int c = t / (si * si), pos = t % (si * si);
    const int y = pos / si, x = pos % si;
    float acc = 0.f;
    if (in_grid(gy0 + y, gx0 + x, n)) {
#pragma unroll
      for (int o = 0; o < COUT; ++o)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            const int yy = y - ky, xx = x - kx;
            if (yy >= 0 && yy < so && xx >= 0 && xx < so)
              acc = fmaf(w[((o * CIN + c) * 3 + ky) * 3 + kx], dz[o * so * so + yy * so + xx], acc);
          }
      acc *= act[t] > 0.f ? 1.f : 0.01f;
    }
    dact[t] = acc;
  }
}

template <int NK>
__global__ void __launch_bounds__(NET_THREADS) k_net_backward(NetBatch batch, const float* __restrict__ dWall,
                                                              const float* __restrict__ params, int bf16,
                                                              float* __restrict__ partials) {
  constexpr int NP = NK == 1 ? MG_NPARAMS : MG_NPARAMS_K3;
  extern __shared__ float sm[];
  float* w = sm;
  float* gw = w + NP;
  float* a0 = gw + NP;
  float* a1 = a0 + 9 * S0 * S0;
  float* a2 = a1 + 7 * S1 * S1;
  float* a3 = a2 + 5 * S2 * S2;
  float* dout = a3 + 3 * S3 * S3;
  float* dz3 = dout + 9 * NK * OT * OT;
  float* dz2 = dz3 + 3 * S3 * S3;
  float* dz1 = dz2 + 5 * S2 * S2;
  NetJob J;
  J.st = batch.st + blockIdx.y * batch.stride;
  J.s = nullptr;
  J.n = batch.n;
  const float* dW = dWall + (size_t)blockIdx.y * batch.stride * NK;
  const int n = J.n;
  const int ntx = (n + OT - 1) / OT;
  const int cta = blockIdx.y * gridDim.x + blockIdx.x;
  float* out = partials + (size_t)cta * NP;
  if ((int)blockIdx.x >= ntx * ntx) {
    for (int t = threadIdx.x; t < NP; t += NET_THREADS) out[t] = 0.f;
    return;
  }
  const int oy = (blockIdx.x / ntx) * OT, ox = (blockIdx.x % ntx) * OT;
  for (int t = threadIdx.x; t < NP; t += NET_THREADS) w[t] = rnd_bf16(params[t], bf16);
  for (int t = threadIdx.x; t < S0 * S0; t += NET_THREADS) {
    const int i = oy - 4 + t / S0, j = ox - 4 + t % S0;
    if (in_grid(i, j, n)) {
      const float d = job_tap(J, 4, i, j);
#pragma unroll
      for (int c = 0; c < 9; ++c) a0[c * S0 * S0 + t] = rnd_bf16(job_tap(J, c, i, j) / d, bf16);
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) a0[c * S0 * S0 + t] = 0.f;
    }
  }
  // dL/d(out) = dW / diag on the tile's outputs (the first kernel; K2, K3 = delta + out)
  const size_t nn = (size_t)n * n;
  for (int t = threadIdx.x; t < 9 * NK * OT * OT; t += NET_THREADS) {
    const int o = t / (OT * OT), pos = t % (OT * OT);
    const int i = oy + pos / OT, j = ox + pos % OT;
    float d = 0.f;
    if (in_grid(i, j, n)) {
      d = dW[o * nn + (size_t)i * n + j];
      if (o < 9) d /= job_tap(J, 4, i, j);
    }
    dout[t] = d;
  }
  __syncthreads();
  conv_layer<9, 7>(w + OFF_W1, a0, S0, a1, S1, oy - 3, ox - 3, n, bf16);
  __syncthreads();
  conv_layer<7, 5>(w + OFF_W2, a1, S1, a2, S2, oy - 2, ox - 2, n, bf16);
  __syncthreads();
  conv_layer<5, 3>(w + OFF_W3, a2, S2, a3, S3, oy - 1, ox - 1, n, bf16);
  __syncthreads();
  conv_wgrad<3, 9 * NK>(dout, OT, a3, S3, gw + OFF_WF);
  conv_igrad<3, 9 * NK>(w + OFF_WF, dout, OT, a3, S3, dz3, oy - 1, ox - 1, n);
  __syncthreads();
  conv_wgrad<5, 3>(dz3, S3, a2, S2, gw + OFF_W3);
  conv_igrad<5, 3>(w + OFF_W3, dz3, S3, a2, S2, dz2, oy - 2, ox - 2, n);
  __syncthreads();
  conv_wgrad<7, 5>(dz2, S2, a1, S1, gw + OFF_W2);
  conv_igrad<7, 5>(w + OFF_W2, dz2, S2, a1, S1, dz1, oy - 3, ox - 3, n);
  __syncthreads();
  conv_wgrad<9, 7>(dz1, S1, a0, S0, gw + OFF_W1);
  __syncthreads();
  for (int t = threadIdx.x; t < NP; t += NET_THREADS) out[t] = gw[t];
}

template <int NP>
__global__ void k_reduce_params(const float* __restrict__ partials, int ncta, float scale, float* __restrict__ g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NP) return;
  float hi = 0.f, lo = 0.f;
  for (int c = 0; c < ncta; ++c) ff_add(hi, lo, partials[(size_t)c * NP + t], 0.f);
  g[t] = scale * (hi + lo);
}

int net_backward_ctas(int n, int nfields) {
  const int ntx = (n + OT - 1) / OT;
  return ntx * ntx * nfields;
}

cudaError_t launch_net_backward(const NetBatch& batch, int nfields, const float* dW, const float* params, int bf16,
                                float* partials, float scale, float* grad, cudaStream_t s) {
  const int ntx = (batch.n + OT - 1) / OT;
  dim3 grid(ntx * ntx, nfields);
  const size_t smem = (size_t)bw_smem_floats<1>() * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_net_backward<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_net_backward<1><<<grid, NET_THREADS, smem, s>>>(batch, dW, params, bf16, partials);
  k_reduce_params<MG_NPARAMS><<<(MG_NPARAMS + 127) / 128, 128, 0, s>>>(partials, ntx * ntx * nfields, scale, grad);
  return cudaGetLastError();
}

cudaError_t launch_net_backward3(const NetBatch& batch, int nfields, const float* dW, const float* params,
                                 float* partials, float scale, float* grad, cudaStream_t s) {
  const int ntx = (batch.n + OT - 1) / OT;
  dim3 grid(ntx * ntx, nfields);
  const size_t smem = (size_t)bw_smem_floats<3>() * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_net_backward<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_net_backward<3><<<grid, NET_THREADS, smem, s>>>(batch, dW, params, 0, partials);
  k_reduce_params<MG_NPARAMS_K3><<<(MG_NPARAMS_K3 + 127) / 128, 128, 0, s>>>(partials, ntx * ntx * nfields, scale,
                                                                              grad);
  return cudaGetLastError();
}

cudaError_t launch_net_forward3_batch(const NetBatch& batch, int nfields, const float* params, float omega,
                                      cudaStream_t s) {
  return fwd_launch<3>(nullptr, batch, nfields, batch.n, params, omega, 0, s);
}

cudaError_t launch_net_forward(const NetJob* jobs_dev, int njobs, int nmax, const float* params, float omega, int bf16,
                               cudaStream_t s) {
  NetBatch none{};
  return fwd_launch<1>(jobs_dev, none, njobs, nmax, params, omega, bf16, s);
}

// The shared-kernel network.  Dense index i of w_k[o][c][t] (k = 1..3) corresponds to the
// shared k_k[o][t]; the last layer wf is common to both layouts.
struct SharedMap {
  int dense, shared, cin;  // start of the layer in each layout; input channels
};
__device__ __forceinline__ SharedMap shared_layer(int i) {
  // dense layer starts: 0, 567, 882, 1017; shared: 0, 63, 108, 135
  if (i < 567) return {0, 0, 9};
  if (i < 882) return {567, 63, 7};
  if (i < 1017) return {882, 108, 5};
  return {1017, 135, 0};
}

__global__ void k_net_expand_shared(const float* __restrict__ shared, float* __restrict__ dense) {
  const float* s = shared + (size_t)blockIdx.y * MG_NPARAMS_SHARED;
  float* d = dense + (size_t)blockIdx.y * MG_NPARAMS;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MG_NPARAMS; i += gridDim.x * blockDim.x) {
    const SharedMap m = shared_layer(i);
    const int j = i - m.dense;
    // conv layers: j = (o * cin + c) * 9 + t  ->  o * 9 + t
    d[i] = s[m.shared + (m.cin ? (j / (9 * m.cin)) * 9 + j % 9 : j)];
  }
}

// grad[k_o[t]] = sum_c dense_grad[w[o][c][t]], c ascending (a fixed order: deterministic)
__global__ void k_net_reduce_shared(const float* __restrict__ gd, float* __restrict__ g) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= MG_NPARAMS_SHARED) return;
  int ds, ss, cin;
  if (q < 63) ds = 0, ss = 0, cin = 9;
  else if (q < 108) ds = 567, ss = 63, cin = 7;
  else if (q < 135) ds = 882, ss = 108, cin = 5;
  else ds = 1017, ss = 135, cin = 0;
  const int j = q - ss;
  if (!cin) {
    g[q] = gd[ds + j];
    return;
  }
  const int o = j / 9, t = j % 9;
  float acc = 0.f;
  for (int c = 0; c < cin; ++c) acc += gd[ds + (o * cin + c) * 9 + t];
  g[q] = acc;
}

cudaError_t launch_net_expand_shared(const float* shared, float* dense, int nsets, cudaStream_t s) {
  k_net_expand_shared<<<dim3((MG_NPARAMS + 255) / 256, nsets), 256, 0, s>>>(shared, dense);
  return cudaGetLastError();
}

cudaError_t launch_net_reduce_shared(const float* dense_grad, float* grad, cudaStream_t s) {
  k_net_reduce_shared<<<(MG_NPARAMS_SHARED + 127) / 128, 128, 0, s>>>(dense_grad, grad);
  return cudaGetLastError();
}

cudaError_t launch_net_forward3(const NetJob* jobs_dev, int njobs, int nmax, const float* params, float omega,
                                cudaStream_t s) {
  NetBatch none{};
  return fwd_launch<3>(jobs_dev, none, njobs, nmax, params, omega, 0, s);
}

cudaError_t launch_net_forward_batch(const NetBatch& batch, int nfields, const float* params, float omega, int bf16,
                                     cudaStream_t s) {
  return fwd_launch<1>(nullptr, batch, nfields, batch.n, params, omega, bf16, s);
}

}  // namespace mg
