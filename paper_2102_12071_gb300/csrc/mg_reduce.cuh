// mg_reduce.cuh -- per-problem norm reduction and the stopping test, shared by the
// residual kernels.
#pragma once
#include "mg_common.cuh"

namespace mg {

// Last-CTA completion of a per-problem sum: every CTA stores its partial; the CTA that
// arrives last adds all partials in float-float and returns true in all its threads.
template <int NTH>
__device__ bool block_partial_and_last(float v, float* partials, unsigned int* counter, int ntiles, int tile,
                                       float& tot_hi, float& tot_lo) {
  __shared__ float wsum[NTH / 32];
  __shared__ bool last;
  __shared__ float fhi[NTH / 32], flo[NTH / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wsum[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int k = 0; k < NTH / 32; ++k) s += wsum[k];
    partials[tile] = s;
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == (unsigned)ntiles - 1u);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  float hi = 0.f, lo = 0.f;
  for (int t = threadIdx.x; t < ntiles; t += NTH) ff_add(hi, lo, __ldcg(partials + t), 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o), olo = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, ohi, olo);
  }
  if (lane == 0) {
    fhi[w] = hi;
    flo[w] = lo;
  }
  __syncthreads();
  hi = 0.f;
  lo = 0.f;
  for (int k = 0; k < NTH / 32; ++k) ff_add(hi, lo, fhi[k], flo[k]);
  tot_hi = hi;
  tot_lo = lo;
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Stopping test after residual evaluation number k = cycles applied so far (Sec. 6.1:
// ||b - A x|| / ||b|| < rtol), with the cycle cap and non-finite residuals.
__device__ __forceinline__ void decide(ProbState& st, float rr_hi, float rr_lo, float rtol, int max_cycles) {
  const int k = __ldcg(&st.iter);
  const float rr = rr_hi + rr_lo, bb = __ldcg(&st.bb_hi) + __ldcg(&st.bb_lo);
  const float rel = sqrtf(rr / bb);
  st.rel = rel;
  st.hist[k % MG_HRING] = rel;
  st.cycles = k;
  st.iter = k + 1;
  if (!isfinite(rel)) {
    st.status = 3;
    st.active = 0;
  } else if (rel < rtol) {
    st.status = 1;
    st.active = 0;
  } else if (k >= max_cycles) {
    st.status = 2;
    st.active = 0;
  }
}

}  // namespace mg
