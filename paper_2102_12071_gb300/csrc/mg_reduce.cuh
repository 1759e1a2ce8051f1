// mg_reduce.cuh -- per-problem norm reduction and the stopping test, shared by the
// residual kernels.
#pragma once
#include "mg_common.cuh"
#include "mg_tma.cuh"

namespace mg {

// Bit pattern of a partial slot not yet written in the current evaluation: a NaN that no
// arithmetic produces (the hardware's NaN is 0x7fffffff).  Slots are filled with it before
// a solve (launch_bnorm) and reset to it by the CTA that consumes them.
constexpr unsigned int kPartialEmpty = 0xffffffffu;

// a load that is performed every time it is executed (never hoisted out of a wait loop)
// and sees stores of other SMs (gpu scope, no stale L1 line)
__device__ __forceinline__ unsigned int ld_relaxed_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Last-CTA completion of a per-problem sum: every CTA stores its partial and counts itself
// with a relaxed atomic; the CTA that arrives last adds all partials in float-float and
// returns true in all its threads.  No CTA fences its store: the last one waits (bounded)
// for each slot to leave the empty pattern instead, so the other CTAs exit without
// waiting for their stores to be acknowledged.
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
    __stcg(partials + tile, s);
    const unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == (unsigned)ntiles - 1u);
  }
  __syncthreads();
  if (!last) return false;
  float hi = 0.f, lo = 0.f;
  unsigned int* slots = reinterpret_cast<unsigned int*>(partials);
  for (int t = threadIdx.x; t < ntiles; t += NTH) {
    // every tile has counted, so its store is issued; it may still be on its way
    unsigned int u = ld_relaxed_gpu(slots + t);
    for (long long it = 0; u == kPartialEmpty && it < kWaitLimit; ++it) u = ld_relaxed_gpu(slots + t);
    ff_add(hi, lo, __uint_as_float(u), 0.f);  // a slot that never arrived stays NaN
    __stcg(slots + t, kPartialEmpty);
  }
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
  if (st.status != 0) st.t_done = global_ns();
}

}  // namespace mg
