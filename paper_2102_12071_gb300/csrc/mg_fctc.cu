// mg_fctc.cu -- inference of the fully connected stencil-to-smoother network (Sec. 4.2,
// parameterisation with fully connected layers; 81 -> 40 -> 40 -> 40 -> 9, Sec. 6.2) on the
// tensor cores, for the bfloat16 mode (weights, inputs and activations in bfloat16, FP32
// accumulation).
//
// A CTA of 128 threads takes tiles of 8 x 16 points; thread t is point t of the tile and
// row t of every layer's M = 128 GEMM.  Per tile:
//   1. the tile's stencils and a one-point halo, each divided by its own diagonal (zero
//      outside the grid), into shared memory;
//   2. row t of the layer-1 operand: the 81 normalised values of the point's 3x3
//      neighbourhood (feature 9 m + c: tap c of neighbour m), bfloat16, padded to K = 96;
//   3. four tcgen05.mma chains, each accumulating in tensor memory (M = 128; N = 48 for the
//      40-unit layers, 16 for the 9 outputs; K in steps of 16), issued by one thread and
//      completed on an mbarrier; between layers each thread reads its accumulator row with
//      tcgen05.ld, applies LeakyReLU(0.01), rounds to bfloat16 and writes the next
//      operand row;
//   4. W = (omega delta_4 + out) / D for the point's 9 taps.
// The weights live in shared memory as the B operands (N x K, K-major), converted once
// per CTA; CTAs loop over the tiles of their job (persistent grid).
#include <cuda_bf16.h>

#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_tc.cuh"
#include "mg_tma.cuh"

namespace mg {

namespace {

constexpr int TM = 128;          // points per tile = MMA M
constexpr int TRW = 8, TCL = 16; // tile rows x columns
constexpr int HR = TRW + 2, HC = TCL + 2;
constexpr int K0 = 96, KH = 48;  // padded K of layer 1 and of the hidden layers
constexpr int NH = 48, NO = 16;  // padded N of the hidden layers and of the output layer
constexpr int IN = 81, HID = 40, OUT = 9;
constexpr int O2 = HID * IN, O3 = O2 + HID * HID, O4 = O3 + HID * HID;
constexpr int TMEM_COLS = 64;
constexpr int FCTC_THREADS = 128;

struct alignas(128) FcTcSmem {
  alignas(128) unsigned char a0[TM * K0 * 2];  // layer-1 operand
  alignas(128) unsigned char ah[TM * KH * 2];  // hidden-layer operand (reused by layers 2..4)
  alignas(128) unsigned char b1[NH * K0 * 2];
  alignas(128) unsigned char b2[NH * KH * 2];
  alignas(128) unsigned char b3[NH * KH * 2];
  alignas(128) unsigned char b4[NO * KH * 2];
  float ns[HR * HC * 9];  // normalised stencils of the tile and its halo, [point][tap]
  uint64_t bar;
  uint32_t tmem;
};

__device__ __forceinline__ float fctc_tap(const float* st, const float* s, int n, int k, int i, int j) {
  if (st) return st[(size_t)k * n * n + (size_t)i * n + j];
  return in_grid(i + k / 3 - 1, j + k % 3 - 1, n) ? s[k] : 0.f;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
  const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
  return lo | (hi << 16);
}

// weight matrix rows x cols (out x in, row-major in params) into a zero-padded N x K operand
__device__ void load_b(unsigned char* dst, const float* w, int rows, int cols, int N, int K) {
  for (int q = threadIdx.x; q < N * K; q += blockDim.x) {
    const int r = q / K, k = q % K;
    const float v = (r < rows && k < cols) ? w[r * cols + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(dst + tc_offset(r, k, K)) = __float2bfloat16_rn(v);
  }
}

// row t of a K-column operand from 8-element groups of values (bfloat16 on the way)
template <int K>
__device__ __forceinline__ void store_row(unsigned char* a, int t, const float* v, int nvalid) {
#pragma unroll
  for (int kc = 0; kc < K / 8; ++kc) {
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (kc * 8 + u < nvalid) ? v[kc * 8 + u] : 0.f;
    uint4 p;
    p.x = pack_bf16(x[0], x[1]);
    p.y = pack_bf16(x[2], x[3]);
    p.z = pack_bf16(x[4], x[5]);
    p.w = pack_bf16(x[6], x[7]);
    *reinterpret_cast<uint4*>(a + tc_offset(t, kc * 8, K)) = p;
  }
}

}  // namespace

// One MMA chain: D = A * B^T over K (steps of 16), then commit to the barrier.
template <int K>
__device__ __forceinline__ void fctc_gemm(uint32_t tmem, const unsigned char* a, const unsigned char* b, uint32_t idesc,
                                          uint64_t* bar) {
  tc_fence_after();
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t ad = tc_sdesc(a + ks * 256, 128, K * 16);
    const uint64_t bd = tc_sdesc(b + ks * 256, 128, K * 16);
    tc_mma(tmem, ad, bd, idesc, ks > 0);
  }
  tc_commit(bar);
}

__global__ void __launch_bounds__(FCTC_THREADS) k_fc_tc(const NetJob* __restrict__ jobs, NetBatch batch,
                                                         const float* __restrict__ params, float omega) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  FcTcSmem& S = *reinterpret_cast<FcTcSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5;
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
  if (warp == 0) tc_alloc(&S.tmem, TMEM_COLS);
  if (t == 0) {
    mbar_init(&S.bar, 1);
    fence_mbar_init();
  }
  load_b(S.b1, params, HID, IN, NH, K0);
  load_b(S.b2, params + O2, HID, HID, NH, KH);
  load_b(S.b3, params + O3, HID, HID, NH, KH);
  load_b(S.b4, params + O4, OUT, HID, NO, KH);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's accumulator lanes
  constexpr uint32_t ID_H = tc_idesc_bf16(TM, NH), ID_O = tc_idesc_bf16(TM, NO);
  const int ntx = (n + TCL - 1) / TCL, nty = (n + TRW - 1) / TRW, ntiles = ntx * nty;
  const size_t nn = (size_t)n * n;
  uint32_t phase = 0;
  bool ok = true;
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int i0 = (tile / ntx) * TRW, j0 = (tile % ntx) * TCL;
    // 1. normalised stencils of the tile and its halo
    for (int q = t; q < HR * HC; q += FCTC_THREADS) {
      const int i = i0 - 1 + q / HC, j = j0 - 1 + q % HC;
      float* o = S.ns + q * 9;
      if (in_grid(i, j, n)) {
        const float d = fctc_tap(st, s, n, 4, i, j);
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = fctc_tap(st, s, n, k, i, j) / d;
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = 0.f;
      }
    }
    __syncthreads();
    // 2. layer-1 operand row t: features 9 m + c of neighbour m of point (ti, tj)
    const int ti = t / TCL, tj = t % TCL;
    {
      float f[IN];
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        const float* nb = S.ns + ((ti + 1 + m / 3 - 1) * HC + (tj + 1 + m % 3 - 1)) * 9;
#pragma unroll
        for (int c = 0; c < 9; ++c) f[9 * m + c] = nb[c];
      }
      store_row<K0>(S.a0, t, f, IN);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // 3. the four layers
    float z[NH];
    for (int layer = 0; layer < 4 && ok; ++layer) {
      if (t == 0) {
        if (layer == 0) fctc_gemm<K0>(tmem, S.a0, S.b1, ID_H, &S.bar);
        else fctc_gemm<KH>(tmem, S.ah, layer == 1 ? S.b2 : layer == 2 ? S.b3 : S.b4, layer == 3 ? ID_O : ID_H,
                           &S.bar);
      }
      // bounded wait for the chain; on expiry a second bounded wait lets it finish before
      // the tensor memory is released, and the tile's outputs become NaN
      const bool done = mbar_wait(&S.bar, phase);
      if (__syncthreads_or(!done)) {
        mbar_wait(&S.bar, phase);
        ok = false;
        break;
      }
      phase ^= 1u;
      tc_fence_after();
      const int ncol = layer == 3 ? NO : NH;
      for (int c = 0; c < ncol; c += 16) {
        float v[16];
        tc_ld16(trow + c, v);
        tc_wait_ld();
#pragma unroll
        for (int u = 0; u < 16; ++u) z[c + u] = v[u];
      }
      if (layer < 3) {
        float a[NH];
#pragma unroll
        for (int o = 0; o < NH; ++o) a[o] = z[o] > 0.f ? z[o] : 0.01f * z[o];
        store_row<KH>(S.ah, t, a, HID);
        fence_async_smem();
      }
      tc_fence_before();
      __syncthreads();
    }
    // 4. the point's kernel
    const int i = i0 + ti, j = j0 + tj;
    if (in_grid(i, j, n)) {
      const float d = fctc_tap(st, s, n, 4, i, j);
      const size_t q = (size_t)i * n + j;
#pragma unroll
      for (int k = 0; k < OUT; ++k) W[k * nn + q] = ok ? ((k == 4 ? omega : 0.f) + z[k]) / d : __int_as_float(0x7fc00000);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------------ launchers
static cudaError_t fctc_prepare(int* ctas_per_sm) {
  static int done[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !done[dev]) {
    e = cudaFuncSetAttribute(k_fc_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FcTcSmem));
    if (e != cudaSuccess) return e;
    // the whole unified L1 as shared memory, so that three CTAs fit on an SM
    e = cudaFuncSetAttribute(k_fc_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = 1;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_fc_tc, FCTC_THREADS, sizeof(FcTcSmem));
}

static cudaError_t fctc_launch(const NetJob* jobs, const NetBatch& batch, int nprob, int nmax, const float* params,
                               float omega, cudaStream_t s) {
  int per_sm = 0, sms = 0, dev = 0;
  cudaError_t e = fctc_prepare(&per_sm);
  if (e != cudaSuccess) return e;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int ntiles = ((nmax + TCL - 1) / TCL) * ((nmax + TRW - 1) / TRW);
  // persistent CTAs: per job as many as shared memory lets stay resident on the GPU (three
  // per SM), at most one per tile of the largest job.  Jobs of different sizes (the levels
  // of a hierarchy) each get that many: a job's CTAs beyond its own tiles exit at once, and
  // the largest job is not left to a share of the GPU while the small ones finish.
  const int fit = (int)((227u * 1024u) / sizeof(FcTcSmem));
  per_sm = per_sm > fit ? per_sm : fit;
  int gx = (per_sm > 0 ? per_sm : 1) * sms;
  gx = gx < 1 ? 1 : (gx > ntiles ? ntiles : gx);
  k_fc_tc<<<dim3(gx, nprob), FCTC_THREADS, sizeof(FcTcSmem), s>>>(jobs, batch, params, omega);
  return cudaGetLastError();
}

cudaError_t launch_fc_forward_tc(const NetJob* jobs_dev, int njobs, int nmax, const float* params, float omega,
                                 cudaStream_t s) {
  NetBatch none = {};
  return fctc_launch(jobs_dev, none, njobs, nmax, params, omega, s);
}

cudaError_t launch_fc_forward_batch_tc(const NetBatch& batch, int nfields, const float* params, float omega,
                                       cudaStream_t s) {
  return fctc_launch(nullptr, batch, nfields, batch.n, params, omega, s);
}

}  // namespace mg
