// mg_common.cuh -- device-side data layout and helpers shared by the sm_103a kernels.
//
// Layout in HBM (all carved from the caller's workspace, 256-byte aligned):
//   per level l, all problems: r_l, e_l            float[nprob][n_l][pitch_l] (128-byte rows)
//   per-point stencil fields (FIELD problems)      float[9][n_l][n_l]
//   per-point smoothing kernels (CNN, FIELD)       float[9][n_l][n_l]
//   kernel class tables (CNN, constant stencils)   float[9][T][T], T = min(n_l, 11)
//   coarsest FP64 inverse                          double[m][m], m = n_L^2
//   ProbDev descriptors, ProbState control blocks, per-CTA norm partials.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define MG_MAXL 14
#define MG_HRING 256          // ring of relative residuals per problem (>= cycles per chunk)
#define MG_TAIL_N 63          // levels at or below this size run in one CTA per problem
#define MG_TAIL_SMEM_MAX (200 * 1024)  // dynamic shared memory limit of the tail kernels
// Levels at or below MG_CT_N run in one CTA cluster per problem, and those at or below
// MG_CT_SOLO in the cluster's first CTA alone (hk: the smoother kind, n0: the finest side).
// On fine grids of side >= 1023 with the network smoothers, whose phases cost more, the
// levels from 63 down with solo levels from 15 measured fastest; Jacobi, and the network
// smoothers on smaller grids (measured at 255), keep band levels from 127 with solo levels
// from 31.
#define MG_CT_N_SHORT 63
#define MG_CT_SOLO_SHORT 15
#define MG_CT_N_LONG 127
#define MG_CT_SOLO_LONG 31
#define MG_CT_SHORT(hk, n0) ((hk) != HK_JACOBI && (n0) >= 1023)
#define MG_CT_N(hk, n0) (MG_CT_SHORT(hk, n0) ? MG_CT_N_SHORT : MG_CT_N_LONG)
#define MG_CT_SOLO(hk, n0) (MG_CT_SHORT(hk, n0) ? MG_CT_SOLO_SHORT : MG_CT_SOLO_LONG)
#ifndef MG_CT_C
#define MG_CT_C 8             // CTAs per cluster (each owns a band of (n + 1) / MG_CT_C rows)
#endif
#define MG_CT_HD 3            // halo rows on each side of a band
#define MG_CT_SMEM_MAX (220 * 1024)    // dynamic shared memory limit of the cluster tail
#define MG_NET_MARGIN 5       // points closer than this to an edge get their own kernel class
#define MG_PROXY (2 * MG_NET_MARGIN + 1)  // proxy grid side for constant-stencil inference
#define MG_NPARAMS 1260
#define MG_NPARAMS_FC 6800  // the fully connected network, 81 -> 40 -> 40 -> 40 -> 9
#define MG_NPARAMS_LIN 54   // the shared-kernel linear smoother of one level: six 3x3 kernels
#define MG_NPARAMS_K3 1746  // the convolutional network with three output kernels (27 outputs)
#define MG_NPARAMS_SHARED 378  // one 3x3 kernel per convolution output channel, then wf

enum { SK_CONST = 0, SK_FIELD = 1 };                 // stencil storage
// layout of the tiled level kernels (mg_tile_shape of mgcnn.h): 32 x 32 tiles (mg_tiles.cu),
// or CTAs of 8 or 4 warp strips of 26 columns over 32 or 64 rows (mg_strip.cu)
enum { MG_SHAPE_TILE32 = 1, MG_SHAPE_STRIP4x32 = 2, MG_SHAPE_STRIP8x64 = 3, MG_SHAPE_STRIP8x32 = 4, MG_SHAPE_PSTRIP = 5 };
// smoother storage: omega/D; per-point kernels of a constant stencil by boundary class;
// per-point kernels of every point; the shared-kernel linear chain (MG_NPARAMS_LIN per level);
// a stack of three per-point kernels of every point ([27][n][n], applied K3(K2(K1 v)))
enum { HK_JACOBI = 0, HK_TABLE = 1, HK_FIELD = 2, HK_LINEAR = 3, HK_STACK3 = 4 };

struct LevelDev {
  int n;
  int T;               // class-table side (HK_TABLE)
  float* r;            // residual / right-hand side of the error equation, [n][pitch]
  float* e;            // correction on this level, [n][pitch]
  float* st;           // SK_FIELD: stencil field [9][n][n]
  float* W;            // HK_TABLE: [9][T][T]; HK_FIELD: [9][n][n]; HK_LINEAR: [6][9], shared;
                       // HK_STACK3: [27][n][n]
  float s[9];          // SK_CONST: stencil of this level (Galerkin product of the finer one)
  int pitch;           // row pitch of r, e and f in floats (multiple of 32: 128-byte rows)
  float* f;            // final correction written by the up-sweep of a tiled level >= 1 (its
                       // e is still read with halos in the same kernel); e elsewhere
};

#define MG_DISPATCH(SKv, HKv, CALL)                                                                        \
  do {                                                                                                     \
    if ((SKv) == SK_CONST && (HKv) == HK_JACOBI) { constexpr int SK_ = SK_CONST, HK_ = HK_JACOBI; CALL; }  \
    else if ((SKv) == SK_CONST && (HKv) == HK_TABLE) { constexpr int SK_ = SK_CONST, HK_ = HK_TABLE; CALL; } \
    else if ((SKv) == SK_FIELD && (HKv) == HK_JACOBI) { constexpr int SK_ = SK_FIELD, HK_ = HK_JACOBI; CALL; } \
    else { constexpr int SK_ = SK_FIELD, HK_ = HK_FIELD; CALL; }                                           \
  } while (0)

// MG_DISPATCH plus the linear smoother and the kernel stack: for the kernels that run every
// smoother kind (the one-CTA coarse tail); the tiled and cluster kernels never see those
#define MG_DISPATCH_T(SKv, HKv, CALL)                                                   \
  do {                                                                                  \
    if ((HKv) == HK_LINEAR) {                                                           \
      if ((SKv) == SK_CONST) { constexpr int SK_ = SK_CONST, HK_ = HK_LINEAR; CALL; }   \
      else { constexpr int SK_ = SK_FIELD, HK_ = HK_LINEAR; CALL; }                     \
    } else if ((HKv) == HK_STACK3) {                                                    \
      if ((SKv) == SK_CONST) { constexpr int SK_ = SK_CONST, HK_ = HK_STACK3; CALL; }   \
      else { constexpr int SK_ = SK_FIELD, HK_ = HK_STACK3; CALL; }                     \
    } else {                                                                            \
      MG_DISPATCH(SKv, HKv, CALL);                                                      \
    }                                                                                   \
  } while (0)

struct ProbDev {
  LevelDev lv[MG_MAXL];
  double* chol;        // coarsest operator, dense FP64 inverse, m x m
  int m;               // n_L^2
  int nu1, nu2;        // smoothing steps before and after the coarse correction (0 read as 1)
  int pad_;
};

struct ProbState {
  float bb_hi, bb_lo;  // ||b||^2 as a float-float pair
  float rel;           // last relative residual
  int active;          // 1 while this problem still iterates
  int iter;            // number of residual evaluations done in this solve
  int cycles;          // V-cycles whose correction has been applied
  int status;          // 0 running, 1 converged, 2 hit max cycles, 3 non-finite residual,
                       // 4 a bounded wait for tile copies expired
  unsigned int counter;  // last-CTA detection for the norm reduction
  int short_wait;        // test setting: nonzero makes the first wait for a tile's copies
                         // give up at once (mg_debug_short_wait); 0 in every normal solve
  int pad_;
  unsigned long long t_start;  // GPU global timer (ns) when the solve's norm of b was formed
  unsigned long long t_done;   // ... when the stopping test ended this problem's iteration
  float hist[MG_HRING];  // hist[k % MG_HRING] = relative residual after k cycles
};

// Control-block fields written by earlier kernels are read through L2 (ld.global.cg).  A
// kernel launched with programmatic serialisation may be resident before those writes
// happen, and a line of the block cached in its SM's L1 by an older kernel would then be
// stale; L2 is the point of coherence, so a .cg load sees the latest value once
// griddepcontrol.wait has returned.
__device__ __forceinline__ int st_active(const ProbState* st) { return __ldcg(&st->active); }

// the GPU's global nanosecond timer (common to all SMs)
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}


// ---------------------------------------------------------------- float-float
// Error-free transformations (Knuth's TwoSum; FMA-based TwoProduct, Dekker 1971).
// Error-free transformations.  Written with the _rn intrinsics, which the compiler never
// contracts into a fused multiply-add: a product feeding one of these sums (a * x in a
// compensated dot product) would otherwise be fused into it, and s + e would no longer
// equal a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// hi + lo -= a (x + xl): one tap of the compensated residual r = b - A x, x = x_hi + x_lo
// (Dot2: exact product and error-free sum for x_hi, plain FP32 for the x_lo term)
__device__ __forceinline__ void dot2_sub(float a, float x, float xl, float& hi, float& lo) {
  const float pr = __fmul_rn(a, x);
  const float pe = fmaf(a, x, -pr);
  float sum, err;
  two_sum(hi, -pr, sum, err);
  hi = sum;
  lo += err - pe;
  lo = fmaf(-a, xl, lo);
}
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bhi, float blo) {
  float s, e;
  two_sum(hi, bhi, s, e);
  e += lo + blo;
  fast_two_sum(s, e, hi, lo);
}

// --------------------------------------------------------------- class tables
// Points at distance >= MG_NET_MARGIN from both edges of a constant-stencil grid see the
// same network input in their whole receptive field, so they share one kernel; nearer
// points get one class per distance.  T = min(n, MG_PROXY); for n <= MG_PROXY the map is
// the identity.
__device__ __forceinline__ int kclass(int i, int n, int T) {
  if (i < MG_NET_MARGIN) return i;
  const int d = n - 1 - i;
  if (d < MG_NET_MARGIN) return T - 1 - d;
  return MG_NET_MARGIN;
}

__device__ __forceinline__ bool in_grid(int i, int j, int n) {
  return (unsigned)i < (unsigned)n && (unsigned)j < (unsigned)n;
}

// warp-level sum
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
