// mg_netfc.cu -- the fully connected stencil-to-smoother network (Sec. 4.2,
// parameterisation with fully connected layers; the four 40-neuron layers of Sec. 6.2).
//
// Per point the input is the 81 stencil values of its 3x3 neighbourhood: feature 9 m + c
// is tap c of the neighbour at offset d_m (m = 3 (di + 1) + (dj + 1)), divided by that
// neighbour's diagonal (the convolutional network's input normalisation), zero outside the
// grid.  Layers 81 -> 40 -> 40 -> 40 -> 9 without biases, LeakyReLU(0.01) after the hidden
// ones; W = (omega * delta_4 + out) / diag.  With bf16, weights, inputs and activations are
// rounded to bfloat16 and products accumulate in FP32.
//
// One thread per point, the 6 800 weights in shared memory (every warp reads the same
// weight at a time: broadcasts).  Training: k_fc_tape recomputes the forward per point and
// records the layer inputs and the back-propagated errors; k_fc_grad sums the weight
// gradients over blocks of points in a fixed order (no atomics: deterministic), and
// k_fc_grad_final adds the blocks in order.
#include <cuda_bf16.h>

#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

constexpr int FC_IN = 81, FC_H = 40, FC_OUT = 9;
constexpr int FC_O2 = FC_H * FC_IN, FC_O3 = FC_O2 + FC_H * FC_H, FC_O4 = FC_O3 + FC_H * FC_H;
static_assert(FC_O4 + FC_OUT * FC_H == MG_NPARAMS_FC, "layer sizes");
constexpr int FC_THREADS = 64;
// tape rows per point (structure of arrays, point index fastest): x, a1, a2, a3, dz1, dz2,
// dz3, dout
constexpr int TP_X = 0, TP_A1 = TP_X + FC_IN, TP_A2 = TP_A1 + FC_H, TP_A3 = TP_A2 + FC_H, TP_D1 = TP_A3 + FC_H,
              TP_D2 = TP_D1 + FC_H, TP_D3 = TP_D2 + FC_H, TP_DO = TP_D3 + FC_H, TP_ROWS = TP_DO + FC_OUT;

__device__ __forceinline__ float fc_rnd(float v, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}
__device__ __forceinline__ float fc_lrelu(float z) { return z > 0.f ? z : 0.01f * z; }

__device__ __forceinline__ float fc_tap(const float* st, const float* s, int n, int k, int i, int j) {
  if (st) return st[(size_t)k * n * n + (size_t)i * n + j];
  return in_grid(i + k / 3 - 1, j + k % 3 - 1, n) ? s[k] : 0.f;
}

__device__ __forceinline__ void fc_load_weights(const float* params, int bf16, float* w) {
  for (int t = threadIdx.x; t < MG_NPARAMS_FC; t += blockDim.x) w[t] = fc_rnd(params[t], bf16);
  __syncthreads();
}

// Layer outputs go to per-thread columns of two shared buffers (hidden unit o of thread t
// at [o * FC_THREADS + t], conflict-free); the outer loops over units stay rolled and only
// the inner products are unrolled, which keeps the code (and its compile time) small.
struct FcSmem {
  float w[MG_NPARAMS_FC];
  float ha[FC_H * FC_THREADS], hb[FC_H * FC_THREADS];
};

// forward of one point to `out`; with a tape, every layer input is stored as it is made
// (rows TP_X, TP_A1, TP_A2, TP_A3 at point column pt)
__device__ __forceinline__ void fc_point(FcSmem& S, const float* st, const float* s, int n, int i, int j, int bf16,
                                         float (&out)[FC_OUT], float* tape, size_t P, size_t pt) {
  const int t = threadIdx.x;
  {
    float x[FC_IN];
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      const int ii = i + m / 3 - 1, jj = j + m % 3 - 1;
      const bool in = in_grid(ii, jj, n);
      const float d = in ? fc_tap(st, s, n, 4, ii, jj) : 1.f;
#pragma unroll
      for (int c = 0; c < 9; ++c) x[9 * m + c] = in ? fc_rnd(fc_tap(st, s, n, c, ii, jj) / d, bf16) : 0.f;
    }
    if (tape) {
      float* r = tape + pt;  // row TP_X = 0; one row of P points further per feature
#pragma unroll
      for (int f = 0; f < FC_IN; ++f, r += P) *r = x[f];
    }
#pragma unroll 1
    for (int o = 0; o < FC_H; ++o) {
      const float* w = S.w + o * FC_IN;
      float acc = 0.f;
#pragma unroll
      for (int f = 0; f < FC_IN; ++f) acc = fmaf(w[f], x[f], acc);
      S.ha[o * FC_THREADS + t] = fc_rnd(fc_lrelu(acc), bf16);
    }
  }
  // hidden layers 2 and 3: ha -> hb -> ha
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    const float* src = (l == 1) ? S.hb : S.ha;
    if (tape) {
      float* r = tape + (TP_A1 + l * FC_H) * P + pt;
#pragma unroll 1
      for (int f = 0; f < FC_H; ++f, r += P) *r = src[f * FC_THREADS + t];
    }
    if (l == 2) break;
    float* dst = (l == 0) ? S.hb : S.ha;
    const float* wl = S.w + (l == 0 ? FC_O2 : FC_O3);
    float h[FC_H];
#pragma unroll
    for (int f = 0; f < FC_H; ++f) h[f] = src[f * FC_THREADS + t];
#pragma unroll 1
    for (int o = 0; o < FC_H; ++o) {
      const float* w = wl + o * FC_H;
      float acc = 0.f;
#pragma unroll
      for (int f = 0; f < FC_H; ++f) acc = fmaf(w[f], h[f], acc);
      dst[o * FC_THREADS + t] = fc_rnd(fc_lrelu(acc), bf16);
    }
  }
  float h[FC_H];
#pragma unroll
  for (int f = 0; f < FC_H; ++f) h[f] = S.ha[f * FC_THREADS + t];
#pragma unroll
  for (int o = 0; o < FC_OUT; ++o) {
    const float* w = S.w + FC_O4 + o * FC_H;
    float acc = 0.f;
#pragma unroll
    for (int f = 0; f < FC_H; ++f) acc = fmaf(w[f], h[f], acc);
    out[o] = acc;
  }
}

// kernels W of one grid (a job: a field, or a constant stencil on a proxy grid) or of a
// uniform batch of fields
__global__ void __launch_bounds__(FC_THREADS) k_fc_forward(const NetJob* __restrict__ jobs, NetBatch batch,
                                                           const float* __restrict__ params, float omega, int bf16) {
  __shared__ FcSmem S;
  fc_load_weights(params, bf16, S.w);
  const float *st, *s;
  float* W;
  int n;
  if (jobs) {
    const NetJob& J = jobs[blockIdx.y];
    st = J.st;
    s = J.s;
    W = J.W;
    n = J.n;
  } else {
    st = batch.st + blockIdx.y * batch.stride;
    s = nullptr;
    W = batch.W + blockIdx.y * batch.stride;
    n = batch.n;
  }
  const int q = blockIdx.x * FC_THREADS + threadIdx.x;
  if (q >= n * n) return;  // after the only barrier
  const int i = q / n, j = q % n;
  float out[FC_OUT];
  fc_point(S, st, s, n, i, j, bf16, out, nullptr, 0, 0);
  const size_t nn = (size_t)n * n;
  const float d = fc_tap(st, s, n, 4, i, j);
#pragma unroll
  for (int k = 0; k < 9; ++k) W[k * nn + q] = ((k == 4 ? omega : 0.f) + out[k]) / d;
}

// per point of a uniform batch: the layer inputs and the errors of dLoss/dW
__global__ void __launch_bounds__(FC_THREADS) k_fc_tape(NetBatch batch, const float* __restrict__ dW,
                                                        const float* __restrict__ params, int bf16,
                                                        float* __restrict__ tape, size_t P) {
  __shared__ FcSmem S;
  fc_load_weights(params, bf16, S.w);
  const int n = batch.n;
  const size_t nn = (size_t)n * n;
  const float* st = batch.st + blockIdx.y * batch.stride;
  const int q = blockIdx.x * FC_THREADS + threadIdx.x;
  if (q >= (int)nn) return;  // after the only barrier
  const int i = q / n, j = q % n, t = threadIdx.x;
  const size_t pt = (size_t)blockIdx.y * nn + q;  // point index of the batch
  float out[FC_OUT];
  fc_point(S, st, nullptr, n, i, j, bf16, out, tape, P, pt);
  const float d = st[4 * nn + q];
  const float* g = dW + blockIdx.y * batch.stride;
  float dout[FC_OUT];
  {
    float* r = tape + TP_DO * P + pt;
#pragma unroll
    for (int k = 0; k < FC_OUT; ++k, r += P) {
      dout[k] = g[k * nn + q] / d;
      *r = dout[k];
    }
  }
  // errors of the hidden layers, back from layer 4, through the thread's shared columns;
  // the masks (LeakyReLU slopes) come from the stored activations (this thread's stores)
  {
    const float* a = tape + TP_A3 * P + pt;
    float* r = tape + TP_D3 * P + pt;
#pragma unroll 1
    for (int f = 0; f < FC_H; ++f, a += P, r += P) {
      float acc = 0.f;
#pragma unroll
      for (int o = 0; o < FC_OUT; ++o) acc = fmaf(S.w[FC_O4 + o * FC_H + f], dout[o], acc);
      const float e = *a > 0.f ? acc : 0.01f * acc;
      S.ha[f * FC_THREADS + t] = e;
      *r = e;
    }
  }
#pragma unroll 1
  for (int l = 0; l < 2; ++l) {
    const float* wl = S.w + (l == 0 ? FC_O3 : FC_O2);
    const float* a = tape + (l == 0 ? TP_A2 : TP_A1) * P + pt;
    float* r = tape + (l == 0 ? TP_D2 : TP_D1) * P + pt;
    const float* src = l == 0 ? S.ha : S.hb;
    float* dst = l == 0 ? S.hb : S.ha;
    float e[FC_H];
#pragma unroll
    for (int o = 0; o < FC_H; ++o) e[o] = src[o * FC_THREADS + t];
#pragma unroll 1
    for (int f = 0; f < FC_H; ++f, a += P, r += P) {
      float acc = 0.f;
#pragma unroll
      for (int o = 0; o < FC_H; ++o) acc = fmaf(wl[o * FC_H + f], e[o], acc);
      const float v = *a > 0.f ? acc : 0.01f * acc;
      dst[f * FC_THREADS + t] = v;
      *r = v;
    }
  }
}

// Weight gradients of one block of FC_CHUNK points for every layer: part[blk][t] =
// sum over the block's points, in order, of err[o] * in[i] (t = the parameter index).
constexpr int FC_CHUNK = 64;
__global__ void __launch_bounds__(256) k_fc_grad(const float* __restrict__ tape, size_t P, float* __restrict__ part) {
  __shared__ float sin_[FC_IN * FC_CHUNK];   // the layer's input rows of the block
  __shared__ float serr[FC_H * FC_CHUNK];    // the layer's error rows
  const size_t p0 = (size_t)blockIdx.x * FC_CHUNK;
  const int np = (int)min((size_t)FC_CHUNK, P - p0);
  float* out = part + (size_t)blockIdx.x * MG_NPARAMS_FC;
  const int rows_in[4] = {TP_X, TP_A1, TP_A2, TP_A3}, rows_err[4] = {TP_D1, TP_D2, TP_D3, TP_DO};
  const int nin[4] = {FC_IN, FC_H, FC_H, FC_H}, nout[4] = {FC_H, FC_H, FC_H, FC_OUT};
  const int off[4] = {0, FC_O2, FC_O3, FC_O4};
  for (int l = 0; l < 4; ++l) {
    for (int t = threadIdx.x; t < nin[l] * FC_CHUNK; t += blockDim.x) {
      const int r = t / FC_CHUNK, c = t % FC_CHUNK;
      sin_[t] = c < np ? tape[(rows_in[l] + r) * P + p0 + c] : 0.f;
    }
    for (int t = threadIdx.x; t < nout[l] * FC_CHUNK; t += blockDim.x) {
      const int r = t / FC_CHUNK, c = t % FC_CHUNK;
      serr[t] = c < np ? tape[(rows_err[l] + r) * P + p0 + c] : 0.f;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nout[l] * nin[l]; t += blockDim.x) {
      const int o = t / nin[l], i = t % nin[l];
      const float* e = serr + o * FC_CHUNK;
      const float* a = sin_ + i * FC_CHUNK;
      float acc = 0.f;
      for (int c = 0; c < np; ++c) acc = fmaf(e[c], a[c], acc);
      out[off[l] + t] = acc;
    }
    __syncthreads();
  }
}

__global__ void k_fc_grad_final(const float* __restrict__ part, int nblk, float scale, float* __restrict__ grad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= MG_NPARAMS_FC) return;
  float hi = 0.f, lo = 0.f;
  for (int b = 0; b < nblk; ++b) ff_add(hi, lo, part[(size_t)b * MG_NPARAMS_FC + t], 0.f);
  grad[t] = scale * (hi + lo);
}

cudaError_t launch_fc_forward(const NetJob* jobs_dev, int njobs, int nmax, const float* params, float omega, int bf16,
                              cudaStream_t s) {
  dim3 grid((nmax * nmax + FC_THREADS - 1) / FC_THREADS, njobs);
  NetBatch none{};
  k_fc_forward<<<grid, FC_THREADS, 0, s>>>(jobs_dev, none, params, omega, bf16);
  return cudaGetLastError();
}

cudaError_t launch_fc_forward_batch(const NetBatch& batch, int nfields, const float* params, float omega, int bf16,
                                    cudaStream_t s) {
  dim3 grid((batch.n * batch.n + FC_THREADS - 1) / FC_THREADS, nfields);
  k_fc_forward<<<grid, FC_THREADS, 0, s>>>(nullptr, batch, params, omega, bf16);
  return cudaGetLastError();
}

size_t fc_backward_floats(int n, int nfields) {
  const size_t P = (size_t)n * n * nfields, nblk = (P + FC_CHUNK - 1) / FC_CHUNK;
  return TP_ROWS * P + nblk * MG_NPARAMS_FC;
}

cudaError_t launch_fc_backward(const NetBatch& batch, int nfields, const float* dW, const float* params, int bf16,
                               float* scratch, float scale, float* grad, cudaStream_t s) {
  const size_t P = (size_t)batch.n * batch.n * nfields;
  const int nblk = (int)((P + FC_CHUNK - 1) / FC_CHUNK);
  float* tape = scratch;
  float* part = scratch + TP_ROWS * P;
  dim3 grid((batch.n * batch.n + FC_THREADS - 1) / FC_THREADS, nfields);
  k_fc_tape<<<grid, FC_THREADS, 0, s>>>(batch, dW, params, bf16, tape, P);
  k_fc_grad<<<nblk, 256, 0, s>>>(tape, P, part);
  k_fc_grad_final<<<(MG_NPARAMS_FC + 127) / 128, 128, 0, s>>>(part, nblk, scale, grad);
  return cudaGetLastError();
}

}  // namespace mg
