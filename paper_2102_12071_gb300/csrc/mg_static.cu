// mg_static.cu -- a solve entry point that allocates no memory at all.
//
// Some callers cannot hand the library a workspace: plugins hosted by a framework whose
// caching allocator owns all device memory (a raw cudaMalloc would bypass its accounting
// or fail inside its pool), control loops with a fixed memory budget that must not risk an
// allocation failure while running, and latency-bound callers that cannot pay for
// cudaMalloc/cudaFree, which may synchronise the whole device.  For them,
// mg_solve_small_static solves small constant-stencil problems with Jacobi-smoothed
// V-cycles using only a fixed scratch array that is part of the library image.
//
// The scratch is one file-scope device array shared by every call on a device and kept
// until the process exits.  Every call looks up its device address on the current device
// (a host-side query, no allocation), so a context rebuilt by cudaDeviceReset between calls
// is seen.  Every call waits for its stream and reads the control blocks back to the host.
// Calls that overlap on the GPU -- from two threads, or on two streams -- race on the array.
#include <math.h>
#include <string.h>

#include "mg_internal.h"
#include "mgcnn.h"

using namespace mg;

namespace {

constexpr size_t kStaticBytes = (size_t)MG_STATIC_SCRATCH_BYTES;

// every field below sits inside g_static_scratch, carved in this order
struct StaticLayout {
  size_t probs, state, partials, xlo, fail, chol, total;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

StaticLayout static_layout(int nprob, int n, int m) {
  StaticLayout L;
  size_t o = 0;
  L.probs = o; o = align256(o + sizeof(ProbDev) * nprob);
  L.state = o; o = align256(o + sizeof(ProbState) * nprob);
  const int nt = tiles_per_side(n);
  L.partials = o; o = align256(o + sizeof(float) * (size_t)nprob * nt * nt);
  L.xlo = o; o = align256(o + sizeof(float) * (size_t)nprob * n * n);
  L.fail = o; o = align256(o + sizeof(int) * 4);
  L.chol = o; o = align256(o + sizeof(double) * (size_t)nprob * m * m);
  L.total = o;
  return L;
}

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[MG_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch on the current device.  In host code the array's
// name is only a host-side stand-in, so the address comes from the runtime on every call.
static mg_status static_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (mg_status)api_fail(MG_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  void* p = nullptr;
  e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
  if (e != cudaSuccess || !p)
    return (mg_status)api_fail(MG_ERR_CUDA, "cudaGetSymbolAddress(g_static_scratch): %s", cudaGetErrorString(e));
  *out = p;
  return MG_OK;
}

#define SCK(call)                                                                                        \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) return (mg_status)api_fail(MG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" mg_status mg_solve_small_static(const mg_problem* problems, int nprob, const mg_options* opts,
                                           const float* b, float* x_hi, float* x_lo, double rtol, int max_cycles,
                                           double* hist, int* cycles, void* stream) {
  if (!problems || !opts || !b || !x_hi) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_solve_small_static: NULL argument");
  if (nprob < 1 || nprob > MG_STATIC_MAX_PROBLEMS)
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_solve_small_static: nprob %d outside 1..%d", nprob,
                               MG_STATIC_MAX_PROBLEMS);
  if (opts->smoother != MG_SMOOTH_JACOBI || opts->nu1 != 1 || opts->nu2 != 1 || opts->coarsest_n != 3)
    return (mg_status)api_fail(MG_ERR_UNSUPPORTED, "mg_solve_small_static: Jacobi V(1,1) to a 3x3 coarsest grid only");
  if (!(opts->omega > 0.f) || !(opts->omega < 2.f))
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_solve_small_static: omega must be in (0, 2)");
  if (max_cycles < 0 || max_cycles > 100000000) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "max_cycles out of range");
  const int n = problems[0].n;
  if (n < 3 || n > MG_STATIC_MAX_N || ((n + 1) & n) != 0)
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_solve_small_static: n = %d must be 2^m - 1 in [3, %d]", n,
                               MG_STATIC_MAX_N);
  for (int p = 0; p < nprob; ++p) {
    const mg_problem& q = problems[p];
    if (q.n != n) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_solve_small_static: problems must share n");
    if (q.kind == MG_PROBLEM_ROTATED) {
      if (!(q.eps > 0.0)) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "problem %d: eps must be > 0", p);
    } else if (q.kind == MG_PROBLEM_STENCIL) {
      if (!q.data) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "problem %d: NULL stencil", p);
    } else {
      return (mg_status)api_fail(MG_ERR_UNSUPPORTED, "mg_solve_small_static: constant-stencil problems only");
    }
  }
  // hierarchy n -> (n-1)/2 -> ... -> 3
  CycleArgs a;
  memset(&a, 0, sizeof(a));
  int L = 0, m = n;
  a.nl[L++] = m;
  while (m > 3) {
    m = (m - 1) / 2;
    a.nl[L++] = m;
  }
  const StaticLayout lay = static_layout(nprob, n, 9);
  if (lay.total > kStaticBytes)
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_solve_small_static: needs %zu bytes of its %zu-byte scratch",
                               lay.total, kStaticBytes);
  void* base = nullptr;
  mg_status st = static_scratch(&base);
  if (st != MG_OK) return st;
  char* sb = (char*)base;
  cudaStream_t s = (cudaStream_t)stream;
  Profiler prof;  // timing stays off: no events are created
  a.probs = (ProbDev*)(sb + lay.probs);
  a.state = (ProbState*)(sb + lay.state);
  a.partials = (float*)(sb + lay.partials);
  a.ntiles_max = tiles_per_side(n) * tiles_per_side(n);
  a.nprob = nprob;
  a.n0 = n;
  a.L = L;
  a.lstar = 0;
  a.sk = SK_CONST;
  a.hk = HK_JACOBI;
  a.nu1 = a.nu2 = 1;
  a.generic = 0;
  a.omega = opts->omega;
  a.stream = s;
  a.prof = &prof;
  // descriptors (level-0 stencils; coarse stencils and the factor are computed on the GPU)
  ProbDev h_probs[MG_STATIC_MAX_PROBLEMS];
  memset(h_probs, 0, sizeof(h_probs));
  for (int p = 0; p < nprob; ++p) {
    ProbDev& d = h_probs[p];
    for (int l = 0; l < L; ++l) {
      d.lv[l].n = a.nl[l];
      d.lv[l].T = a.nl[l] < MG_PROXY ? a.nl[l] : MG_PROXY;
    }
    d.m = 9;
    d.chol = (double*)(sb + lay.chol) + (size_t)p * 81;
    if (problems[p].kind == MG_PROBLEM_ROTATED) {
      if (mg_rotated_stencil(problems[p].eps, problems[p].theta, d.lv[0].s) != MG_OK) return MG_ERR_INVALID_ARG;
    } else {
      for (int k = 0; k < 9; ++k) d.lv[0].s[k] = problems[p].data[k];
    }
    if (!(d.lv[0].s[4] > 0.f)) return (mg_status)api_fail(MG_ERR_INVALID_ARG, "problem %d: diagonal must be > 0", p);
  }
  int* d_fail = (int*)(sb + lay.fail);
  SCK(cudaMemcpyAsync(a.probs, h_probs, sizeof(ProbDev) * nprob, cudaMemcpyHostToDevice, s));
  SCK(cudaMemsetAsync(d_fail, 0, sizeof(int), s));
  SCK(launch_rap_const(a.probs, nprob, L, s));
  SCK(launch_coarsest_factor(a.probs, nprob, L, SK_CONST, d_fail, s));
  float* xlo = x_lo;
  if (!xlo) {
    xlo = (float*)(sb + lay.xlo);
    SCK(cudaMemsetAsync(xlo, 0, sizeof(float) * (size_t)nprob * n * n, s));
  }
  // the control blocks keep the previous call's contents: start from zero
  SCK(cudaMemsetAsync(a.state, 0, sizeof(ProbState) * nprob, s));
  SCK(launch_bnorm(a, b));
  int failed = 0;
  SCK(cudaMemcpyAsync(&failed, d_fail, sizeof(int), cudaMemcpyDeviceToHost, s));
  SCK(cudaStreamSynchronize(s));
  if (failed) return (mg_status)api_fail(MG_ERR_NUMERIC, "coarsest operator is not positive definite");
  ProbState h_state[MG_STATIC_MAX_PROBLEMS];
  int seen[MG_STATIC_MAX_PROBLEMS] = {0};
  const float frtol = (float)rtol;
  int G = 16;
  for (;;) {
    SCK(launch_tail_solve(a, b, x_hi, xlo, frtol, max_cycles, G, 0));
    SCK(cudaMemcpyAsync(h_state, a.state, sizeof(ProbState) * nprob, cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    int active = 0;
    for (int p = 0; p < nprob; ++p) {
      const ProbState& S = h_state[p];
      if (hist)
        for (int k = seen[p]; k < S.iter; ++k) hist[(size_t)p * (max_cycles + 1) + k] = S.hist[k % MG_HRING];
      seen[p] = S.iter;
      active += S.active;
    }
    if (!active) break;
    G = G < 128 ? 2 * G : 128;
  }
  mg_status rc = MG_OK;
  for (int p = 0; p < nprob; ++p) {
    if (cycles) cycles[p] = h_state[p].cycles;
    if (h_state[p].status == 3) rc = MG_ERR_NUMERIC;
    else if (h_state[p].status == 2 && rc == MG_OK) rc = MG_ERR_NOT_CONVERGED;
  }
  if (rc == MG_ERR_NUMERIC) api_fail(rc, "non-finite residual");
  else if (rc == MG_ERR_NOT_CONVERGED) api_fail(rc, "max_cycles reached before rtol");
  return rc;
}
