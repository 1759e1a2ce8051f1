// mg_tile.cuh -- pieces shared by the tiled level kernels: the 3x3 register window a
// thread slides down a strip of a shared-memory tile, the stencil sum over it, and the
// bounded wait for a tile's copies.
#pragma once
#include "mg_common.cuh"
#include "mg_tma.cuh"

namespace mg {

// 3x3 neighbourhood of a point in registers: rows above (a), at (b) and below (c) it,
// columns left (0), centre (1) and right (2); tap k = 3*(di+1) + (dj+1) of a stencil
// multiplies a0 a1 a2 b0 b1 b2 c0 c1 c2 in that order.
struct Win {
  float a0, a1, a2, b0, b1, b2, c0, c1, c2;
  __device__ __forceinline__ void load_ab(const float* c, int ts) {
    a0 = c[-ts - 1]; a1 = c[-ts]; a2 = c[-ts + 1];
    b0 = c[-1]; b1 = c[0]; b2 = c[1];
  }
  __device__ __forceinline__ void load_c(const float* c, int ts) {
    c0 = c[ts - 1]; c1 = c[ts]; c2 = c[ts + 1];
  }
  __device__ __forceinline__ void shift() {
    a0 = b0; a1 = b1; a2 = b2;
    b0 = c0; b1 = c1; b2 = c2;
  }
};

// sum of w_k v_k, centre first (the order of stencil_apply)
__device__ __forceinline__ float dot9(const float (&w)[9], const Win& v) {
  float acc = w[4] * v.b1;
  acc = fmaf(w[0], v.a0, acc);
  acc = fmaf(w[1], v.a1, acc);
  acc = fmaf(w[2], v.a2, acc);
  acc = fmaf(w[3], v.b0, acc);
  acc = fmaf(w[5], v.b2, acc);
  acc = fmaf(w[6], v.c0, acc);
  acc = fmaf(w[7], v.c1, acc);
  acc = fmaf(w[8], v.c2, acc);
  return acc;
}

// Waits for the CTA's copies; on expiry marks the problem timed out (status 4) and waits
// once more, with the full bound, for copies still in flight, so that none is outstanding
// when the CTA exits.  Returns false in every thread then.  With the test setting
// st.short_wait the first wait gives up without polling (the expiry path on demand).
__device__ __forceinline__ bool tile_wait(uint64_t* bar, ProbState& st) {
  const bool ok = __ldcg(&st.short_wait) == 0 && mbar_wait(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      st.status = 4;
      st.active = 0;
    }
    mbar_wait(bar, 0);
    return false;
  }
  return true;
}

// tile_wait for a barrier in use more than once (the completion of phase `parity`); on
// expiry it also drains the copies in flight on `other` (phase other_parity), if any
__device__ __forceinline__ bool tile_wait_phase(uint64_t* bar, uint32_t parity, uint64_t* other, uint32_t other_parity,
                                                ProbState& st) {
  const bool ok = __ldcg(&st.short_wait) == 0 && mbar_wait(bar, parity);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      st.status = 4;
      st.active = 0;
    }
    mbar_wait(bar, parity);
    if (other) mbar_wait(other, other_parity);
    return false;
  }
  return true;
}

}  // namespace mg
