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

// jobs == nullptr: job y is field y of a uniform batch (batch.st/W + y * batch.stride)
__global__ void __launch_bounds__(NET_THREADS) k_net_forward(const NetJob* __restrict__ jobs, NetBatch batch,
                                                             const float* __restrict__ params, float omega,
                                                             int bf16) {
  __shared__ float w[MG_NPARAMS];
  __shared__ float bufA[9 * S0 * S0];   // a0, later a2
  __shared__ float bufB[7 * S1 * S1];   // a1, later a3
  NetJob J;
  if (jobs) {
    J = jobs[blockIdx.y];
  } else {
    J.st = batch.st + blockIdx.y * batch.stride;
    J.s = nullptr;
    J.W = batch.W + blockIdx.y * batch.stride;
    J.n = batch.n;
  }
  const int n = J.n;
  const int ntx = (n + OT - 1) / OT;
  if ((int)blockIdx.x >= ntx * ntx) return;
  const int oy = (blockIdx.x / ntx) * OT, ox = (blockIdx.x % ntx) * OT;
  for (int t = threadIdx.x; t < MG_NPARAMS; t += NET_THREADS) w[t] = rnd_bf16(params[t], bf16);
  // a0: normalised stencil on rows/cols [oy-4, oy+OT+4)
  for (int t = threadIdx.x; t < S0 * S0; t += NET_THREADS) {
    const int i = oy - 4 + t / S0, j = ox - 4 + t % S0;
    if (in_grid(i, j, n)) {
      const float d = job_tap(J, 4, i, j);
#pragma unroll
      for (int c = 0; c < 9; ++c) bufA[c * S0 * S0 + t] = rnd_bf16(job_tap(J, c, i, j) / d, bf16);
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) bufA[c * S0 * S0 + t] = 0.f;
    }
  }
  __syncthreads();
  conv_layer<9, 7>(w + OFF_W1, bufA, S0, bufB, S1, oy - 3, ox - 3, n, bf16);
  __syncthreads();
  conv_layer<7, 5>(w + OFF_W2, bufB, S1, bufA, S2, oy - 2, ox - 2, n, bf16);
  __syncthreads();
  conv_layer<5, 3>(w + OFF_W3, bufA, S2, bufB, S3, oy - 1, ox - 1, n, bf16);
  __syncthreads();
  // output layer over the 3x3 window of the 3-channel map
  const size_t nn = (size_t)n * n;
  for (int t = threadIdx.x; t < 9 * OT * OT; t += NET_THREADS) {
    const int o = t / (OT * OT), pos = t % (OT * OT);
    const int y = pos / OT, x = pos % OT;
    const int i = oy + y, j = ox + x;
    if (!in_grid(i, j, n)) continue;
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx)
          acc = fmaf(w[OFF_WF + ((o * 3 + c) * 3 + ky) * 3 + kx], bufB[c * S3 * S3 + (y + ky) * S3 + x + kx], acc);
    const float d = job_tap(J, 4, i, j);
    J.W[o * nn + (size_t)i * n + j] = ((o == 4 ? omega : 0.f) + acc) / d;
  }
}

cudaError_t launch_net_forward(const NetJob* jobs_dev, int njobs, int nmax, const float* params, float omega, int bf16,
                               cudaStream_t s) {
  const int ntx = (nmax + OT - 1) / OT;
  dim3 grid(ntx * ntx, njobs);
  NetBatch none{};
  k_net_forward<<<grid, NET_THREADS, 0, s>>>(jobs_dev, none, params, omega, bf16);
  return cudaGetLastError();
}

cudaError_t launch_net_forward_batch(const NetBatch& batch, int nfields, const float* params, float omega, int bf16,
                                     cudaStream_t s) {
  const int ntx = (batch.n + OT - 1) / OT;
  dim3 grid(ntx * ntx, nfields);
  k_net_forward<<<grid, NET_THREADS, 0, s>>>(nullptr, batch, params, omega, bf16);
  return cudaGetLastError();
}

}  // namespace mg
