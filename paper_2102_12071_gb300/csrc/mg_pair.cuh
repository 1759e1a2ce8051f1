// mg_pair.cuh -- two adjacent grid columns per thread in packed FP32.
//
// A pair's two values share one 64-bit register pair and each arithmetic step is one
// packed instruction (add, mul, fma on .f32x2: __fadd2_rn, __fmul2_rn, __ffma2_rn), each
// lane rounded exactly as the scalar instruction, so error-free transformations stay exact
// lane by lane.  A 3x3 window row around the pair (c, c+1) is the four columns c-1 .. c+2.
// A 64-bit shared-memory access is served per half-warp: a half-warp that takes 16
// consecutive pairs of one row touches each bank once.
#pragma once
#include <cuda_runtime.h>

#include "mg_tile.cuh"

namespace mg {

__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 ng2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, ng2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  e = sub2(b, sub2(s, a));
}
// dot2_sub on a pair: hi + lo -= a (x + xl)
__device__ __forceinline__ void dot2_sub2(float a, float2 x, float2 xl, float2& hi, float2& lo) {
  const float2 pr = mul2(p2(a), x);
  const float2 pe = fma2(p2(a), x, ng2(pr));
  float2 sum, err;
  two_sum2(hi, ng2(pr), sum, err);
  hi = sum;
  lo = add2(lo, sub2(err, pe));
  lo = fma2(p2(-a), xl, lo);
}

// Three rows of the columns c-1 .. c+2 around the pair (c, c+1): l = (c-1, c), m = (c, c+1),
// r = (c+1, c+2) of rows a, b, c, the left, centre and right operands of the pair's stencil.
struct Win2 {
  float2 la, ma, ra, lb, mb, rb, lc, mc, rc;
  __device__ __forceinline__ void shift() {
    la = lb; ma = mb; ra = rb;
    lb = lc; mb = mc; rb = rc;
  }
};
// one window row; p points at column c-1, which is even (c odd): two aligned loads
__device__ __forceinline__ void row_odd(const float* p, float2& l, float2& m, float2& r) {
  const float2 u = ld2(p), w = ld2(p + 2);
  l = u;
  r = w;
  m = make_float2(u.y, w.x);
}
// one window row; p points at column c, which is even: one aligned and two single loads
__device__ __forceinline__ void row_even(const float* p, float2& l, float2& m, float2& r) {
  const float2 u = ld2(p);
  const float a = p[-1], b = p[2];
  l = make_float2(a, u.x);
  m = u;
  r = make_float2(u.y, b);
}
// Sum of w_k v_k for both points, centre first (the order of dot9), without building the
// pairs that are not already in a register pair.  For
// a window from row_odd, l and r are the loaded pairs and m = (l.y, r.x): its three taps run
// as two scalar FMAs each.  For a window from row_even, m is the loaded pair and the outer
// columns c-1 = l.x and c+2 = r.y are single registers: l = (l.x, m.x) and r = (m.y, r.y)
// run as scalar FMAs.  Each lane performs the same operations in the same order as dot9.
template <bool ODD>
__device__ __forceinline__ float2 dot9w(const float (&w)[9], const Win2& v) {
  float2 acc;
  auto tap = [&](float wk, const float2& l, const float2& m, const float2& r, int col) {
    // col 0: left (c-1, c), 1: centre (c, c+1), 2: right (c+1, c+2)
    if (ODD) {
      if (col == 0) acc = fma2(p2(wk), l, acc);
      else if (col == 2) acc = fma2(p2(wk), r, acc);
      else {
        acc.x = fmaf(wk, l.y, acc.x);
        acc.y = fmaf(wk, r.x, acc.y);
      }
    } else {
      if (col == 1) acc = fma2(p2(wk), m, acc);
      else if (col == 0) {
        acc.x = fmaf(wk, l.x, acc.x);
        acc.y = fmaf(wk, m.x, acc.y);
      } else {
        acc.x = fmaf(wk, m.y, acc.x);
        acc.y = fmaf(wk, r.y, acc.y);
      }
    }
  };
  if (ODD) acc = make_float2(w[4] * v.lb.y, w[4] * v.rb.x);
  else acc = mul2(p2(w[4]), v.mb);
  tap(w[0], v.la, v.ma, v.ra, 0);
  tap(w[1], v.la, v.ma, v.ra, 1);
  tap(w[2], v.la, v.ma, v.ra, 2);
  tap(w[3], v.lb, v.mb, v.rb, 0);
  tap(w[5], v.lb, v.mb, v.rb, 2);
  tap(w[6], v.lc, v.mc, v.rc, 0);
  tap(w[7], v.lc, v.mc, v.rc, 1);
  tap(w[8], v.lc, v.mc, v.rc, 2);
  return acc;
}
// A window row around the pair (c, c+1) as the pair and its two outer columns: l = c-1,
// m = (c, c+1), r = c+2 (a row of the warp-strip kernels, whose neighbours come from the
// adjacent lanes).
struct PRow {
  float l;
  float2 m;
  float r;
};
// the window of three such rows in the form dot9w<false> reads (l.x, m, r.y)
__device__ __forceinline__ Win2 win_rows(const PRow& a, const PRow& b, const PRow& c) {
  Win2 v;
  v.la = make_float2(a.l, a.m.x); v.ma = a.m; v.ra = make_float2(a.m.y, a.r);
  v.lb = make_float2(b.l, b.m.x); v.mb = b.m; v.rb = make_float2(b.m.y, b.r);
  v.lc = make_float2(c.l, c.m.x); v.mc = c.m; v.rc = make_float2(c.m.y, c.r);
  return v;
}
// dot9w<false> with a kernel of its own for each column of the pair (w[k].x for column c,
// w[k].y for c+1): each lane performs the operations of dot9 in its order
__device__ __forceinline__ float2 dot9wp(const float2 (&w)[9], const Win2& v) {
  float2 acc = mul2(w[4], v.mb);
  auto tap = [&](const float2& wk, const float2& l, const float2& m, const float2& r, int col) {
    if (col == 1) acc = fma2(wk, m, acc);
    else if (col == 0) {
      acc.x = fmaf(wk.x, l.x, acc.x);
      acc.y = fmaf(wk.y, m.x, acc.y);
    } else {
      acc.x = fmaf(wk.x, m.y, acc.x);
      acc.y = fmaf(wk.y, r.y, acc.y);
    }
  };
  tap(w[0], v.la, v.ma, v.ra, 0);
  tap(w[1], v.la, v.ma, v.ra, 1);
  tap(w[2], v.la, v.ma, v.ra, 2);
  tap(w[3], v.lb, v.mb, v.rb, 0);
  tap(w[5], v.lb, v.mb, v.rb, 2);
  tap(w[6], v.lc, v.mc, v.rc, 0);
  tap(w[7], v.lc, v.mc, v.rc, 1);
  tap(w[8], v.lc, v.mc, v.rc, 2);
  return acc;
}
// the scalar window of one point of the pair (lane 0: column c, lane 1: column c+1)
__device__ __forceinline__ Win lane_win(const Win2& v, int lane) {
  Win w;
  w.a0 = lane ? v.la.y : v.la.x; w.a1 = lane ? v.ma.y : v.ma.x; w.a2 = lane ? v.ra.y : v.ra.x;
  w.b0 = lane ? v.lb.y : v.lb.x; w.b1 = lane ? v.mb.y : v.mb.x; w.b2 = lane ? v.rb.y : v.rb.x;
  w.c0 = lane ? v.lc.y : v.lc.x; w.c1 = lane ? v.mc.y : v.mc.x; w.c2 = lane ? v.rc.y : v.rc.x;
  return w;
}
// Work item of thread t in a phase over NQ pairs and NS row strips: pairs 0 .. 15 first, one
// strip per half-warp (16 consecutive pairs of a row: conflict-free 64-bit shared accesses),
// then pairs 16 .. NQ-1 of every strip; false for the threads left idle.
template <int NQ, int NS>
__device__ __forceinline__ bool chunk_item(int t, int& q, int& strip) {
  if (t < 16 * NS) {
    q = t & 15;
    strip = t >> 4;
    return true;
  }
  if constexpr (NQ > 16) {
    t -= 16 * NS;
    if (t < (NQ - 16) * NS) {
      q = 16 + t % (NQ - 16);
      strip = t / (NQ - 16);
      return true;
    }
  }
  return false;
}

}  // namespace mg
