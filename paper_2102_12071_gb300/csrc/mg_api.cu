// mg_api.cu -- host side of the C ABI declared in include/mgcnn.h.
//
// Validates arguments, carves the caller's workspace, records the device descriptors of
// the hierarchy and queues the kernels of mg_setup.cu, mg_cycle.cu and mg_net.cu on the
// caller's stream.  It never allocates device memory and never aborts.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "mg_internal.h"
#include "mgcnn.h"

using namespace mg;

static thread_local char g_err[512] = "";

static mg_status fail(mg_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

int mg::api_fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return status;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(MG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));  \
  } while (0)

// ------------------------------------------------------------------ planning
namespace {

struct Plan {
  int nprob = 0, n0 = 0, L = 0, lstar = 0, sk = SK_CONST, hk = HK_JACOBI, tail_solve = 0;
  int ctail = 0;    // levels >= lstar in one CTA cluster per problem
  int generic = 0;  // levels above the tail in batched level kernels (mg_linear.cu)
  int nu1 = 1, nu2 = 1;
  int lstar1 = 0;   // first level of the one-CTA tail (the fallback of the cluster tail)
  int shape = MG_SHAPE_PSTRIP;  // layout of the tiled level kernels
  int nl[MG_MAXL] = {0};
  int ntiles_max = 0;
  size_t bytes = 0;
};

bool is_pow2m1(int n) { return n >= 1 && ((n + 1) & n) == 0; }

mg_status make_plan(const mg_problem* probs, int nprob, const mg_options* o, Plan& P) {
  if (!probs || nprob <= 0 || !o) return fail(MG_ERR_INVALID_ARG, "problems/options missing or nprob <= 0");
  if (nprob > 65535) return fail(MG_ERR_INVALID_ARG, "nprob %d > 65535", nprob);
  if (o->smoother != MG_SMOOTH_JACOBI && o->smoother != MG_SMOOTH_CNN)
    return fail(MG_ERR_INVALID_ARG, "unknown smoother %d", o->smoother);
  if (o->nu1 < 1 || o->nu2 < 1 || o->nu1 > 8 || o->nu2 > 8)
    return fail(MG_ERR_INVALID_ARG, "nu1 and nu2 must be in [1, 8]");
  if ((o->nu1 != 1 || o->nu2 != 1) && !(o->smoother == MG_SMOOTH_JACOBI ||
                                        (o->smoother == MG_SMOOTH_CNN && o->net_arch == MG_NET_LINEAR)))
    return fail(MG_ERR_UNSUPPORTED, "nu1, nu2 > 1 need the Jacobi or the linear smoother");
  if (o->coarsest_n != 3 && o->coarsest_n != 7) return fail(MG_ERR_UNSUPPORTED, "coarsest_n must be 3 or 7");
  if (!(o->omega > 0.f) || !(o->omega < 2.f)) return fail(MG_ERR_INVALID_ARG, "omega must be in (0, 2)");
  if (o->net_levels < 0 || o->net_levels > MG_MAXL) return fail(MG_ERR_INVALID_ARG, "net_levels out of range");
  if (o->net_arch != MG_NET_CONV && o->net_arch != MG_NET_FC && o->net_arch != MG_NET_LINEAR &&
      o->net_arch != MG_NET_CONV3 && o->net_arch != MG_NET_CONV_SHARED)
    return fail(MG_ERR_INVALID_ARG, "unknown net_arch");
  if (o->smoother == MG_SMOOTH_CNN && o->net_arch == MG_NET_CONV3 && o->conv_bf16)
    return fail(MG_ERR_UNSUPPORTED, "the three-kernel network runs in FP32");
  if (o->net_per_problem != 0 && o->net_per_problem != 1) return fail(MG_ERR_INVALID_ARG, "net_per_problem must be 0 or 1");
  if (o->tile_shape < MG_TILE_DEFAULT || o->tile_shape > MG_TILE_PSTRIP)
    return fail(MG_ERR_INVALID_ARG, "unknown tile_shape %d", o->tile_shape);
  P.shape = o->tile_shape == MG_TILE_DEFAULT ? MG_SHAPE_PSTRIP : o->tile_shape;
  if (o->net_per_problem && !(o->smoother == MG_SMOOTH_CNN && o->net_arch == MG_NET_LINEAR))
    return fail(MG_ERR_UNSUPPORTED, "per-problem parameter sets need the linear smoother (MG_NET_LINEAR)");
  const int n = probs[0].n;
  if (!is_pow2m1(n) || n < o->coarsest_n || n > 8191)
    return fail(MG_ERR_INVALID_ARG, "n = %d must be 2^m - 1 in [coarsest_n, 8191]", n);
  int nconst = 0;
  for (int p = 0; p < nprob; ++p) {
    const mg_problem& q = probs[p];
    if (q.n != n) return fail(MG_ERR_UNSUPPORTED, "all problems of a batch must share n (problem %d)", p);
    switch (q.kind) {
      case MG_PROBLEM_ROTATED:
        if (!(q.eps > 0.0) || !isfinite(q.theta)) return fail(MG_ERR_INVALID_ARG, "problem %d: eps must be > 0", p);
        ++nconst;
        break;
      case MG_PROBLEM_STENCIL:
        if (!q.data) return fail(MG_ERR_INVALID_ARG, "problem %d: stencil pointer is NULL", p);
        ++nconst;
        break;
      case MG_PROBLEM_VARCOEF5:
      case MG_PROBLEM_FIELD:
        if (!q.data) return fail(MG_ERR_INVALID_ARG, "problem %d: device data pointer is NULL", p);
        break;
      default:
        return fail(MG_ERR_INVALID_ARG, "problem %d: unknown kind %d", p, q.kind);
    }
  }
  if (nconst != 0 && nconst != nprob)
    return fail(MG_ERR_UNSUPPORTED, "a batch mixes constant-stencil and per-point problems");
  P.nprob = nprob;
  P.n0 = n;
  P.sk = nconst ? SK_CONST : SK_FIELD;
  P.hk = o->smoother == MG_SMOOTH_JACOBI ? HK_JACOBI
         : o->net_arch == MG_NET_LINEAR  ? HK_LINEAR
         : o->net_arch == MG_NET_CONV3   ? HK_STACK3
                                         : (P.sk == SK_CONST ? HK_TABLE : HK_FIELD);
  // the paired strips cover constant stencils with Jacobi or network kernels; other
  // smoothers keep the 32 x 32 tiles
  if (P.shape == MG_SHAPE_PSTRIP && !(P.sk == SK_CONST && (P.hk == HK_JACOBI || P.hk == HK_TABLE)))
    P.shape = MG_SHAPE_TILE32;
  if (o->smoother_transpose && P.hk == HK_TABLE)
    return fail(MG_ERR_UNSUPPORTED, "smoother_transpose needs per-point problems (kinds VARCOEF5, FIELD)");
  int m = n, L = 0;
  P.nl[L++] = m;
  while (m > o->coarsest_n) {
    m = (m - 1) / 2;
    if (L >= MG_MAXL) return fail(MG_ERR_INVALID_ARG, "too many levels");
    P.nl[L++] = m;
  }
  P.L = L;
  P.lstar = 0;
  while (P.lstar < L && P.nl[P.lstar] > MG_TAIL_N) ++P.lstar;
  P.lstar1 = P.lstar;
  P.tail_solve = P.lstar == 0;
  P.nu1 = o->nu1;
  P.nu2 = o->nu2;
  P.generic = P.hk == HK_LINEAR || P.hk == HK_STACK3 || P.nu1 != 1 || P.nu2 != 1;
  const int nt = tiles_per_side(n);
  P.ntiles_max = nt * nt;
  if (tail_smem_bytes(P.nl, P.lstar, L, P.hk) > MG_TAIL_SMEM_MAX)
    return fail(MG_ERR_UNSUPPORTED, "tail does not fit in shared memory");
  if (!P.tail_solve && o->cluster_tail && !P.generic) {
    int ls = 1;  // the finest level stays tiled: it carries the outer residual and update
    while (ls < L && P.nl[ls] > MG_CT_N(P.hk, P.nl[0])) ++ls;
    if (ls < L && P.nl[ls] > MG_CT_SOLO(P.hk, P.nl[0]) && ctail_smem_bytes(P.nl, ls, L, P.hk) <= MG_CT_SMEM_MAX) {
      P.lstar = ls;
      P.ctail = 1;
    }
  }
  return MG_OK;
}

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

}  // namespace

struct mg_ctx {
  Plan plan;
  mg_options opts;
  CycleArgs args;
  std::vector<ProbDev> h_probs;
  ProbState* h_state = nullptr;  // pinned host copy of the control blocks (nprob entries)
  float* xlo_ws = nullptr;
  int* d_fail = nullptr;
  NetJob* d_jobs = nullptr;
  int* d_active = nullptr;      // compacted list of problems still iterating
  float* tscratch = nullptr;    // kernel transposition scratch (smoother_transpose)
  float* lin = nullptr;         // the linear smoother's weights, [L-1][MG_NPARAMS_LIN]
  float* net_dense = nullptr;   // MG_NET_CONV_SHARED: its sets in the dense layout
  LinMaps lin_maps;             // its tensor maps (levels above the tail)
  std::vector<int> h_active;
  LevelArrays arrays;
  TileMaps maps;
  Profiler prof;
  // captured cycles (every level kernel; the last one ends with the new residual and the
  // stopping test) per compacted launch size
  struct CycleGraph {
    int nactive, max_cycles;
    float rtol;
    cudaGraphExec_t exec;
    long long nodes;
  };
  std::vector<CycleGraph> graphs;
  cudaStream_t capture_stream = nullptr;
  ~mg_ctx() {
    for (CycleGraph& g : graphs) cudaGraphExecDestroy(g.exec);
    if (h_state) cudaFreeHost(h_state);
    if (capture_stream) cudaStreamDestroy(capture_stream);
  }
};

// cycles per executable graph; every chunk of the solve loop is a multiple of it
constexpr int kGraphCycles = 16;

// The executable graph of kGraphCycles cycles for the current launch size, captured on a
// private stream the first time it is needed and replayed on the caller's stream afterwards.
static mg_status cycle_graph(mg_ctx* ctx, const CycleArgs& a, float rtol, int max_cycles, cudaGraphExec_t* out,
                             long long* nodes) {
  const int nact = a.active ? a.nactive : 0;
  for (const mg_ctx::CycleGraph& g : ctx->graphs)
    if (g.nactive == nact && g.rtol == rtol && g.max_cycles == max_cycles) {
      *out = g.exec;
      *nodes = g.nodes;
      return MG_OK;
    }
  if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  CK(prepare_tail(a));
  CycleArgs c = a;
  c.stream = ctx->capture_stream;
  c.pdl = true;
  const long long before = ctx->prof.launches;
  CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e2 = cudaSuccess;
  for (int k = 0; k < kGraphCycles && e2 == cudaSuccess; ++k) {
    e2 = launch_cycle(c, rtol, max_cycles, k & 1);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(c.stream, &graph);
  if (e2 != cudaSuccess || e3 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(MG_ERR_CUDA, "capturing the cycle graph: %s", cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
  }
  cudaGraphExec_t exec = nullptr;
  cudaError_t e4 = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e4 != cudaSuccess) return fail(MG_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e4));
  mg_ctx::CycleGraph g;
  g.nactive = nact;
  g.rtol = rtol;
  g.max_cycles = max_cycles;
  g.exec = exec;
  g.nodes = ctx->prof.launches - before;
  ctx->prof.launches = before;
  ctx->graphs.push_back(g);
  *out = exec;
  *nodes = g.nodes;
  return MG_OK;
}

// Cycles of the next chunk of the solve loop.  Launches cover the problems active at the
// start of a chunk, so a problem converging inside it keeps launching (idle) CTAs until
// the chunk ends: the chunk is sized to end when the next problem is expected to reach
// rtol at its recent convergence rate, as a multiple of the graph length and at most one
// ring of residual history; without a rate estimate it doubles.
static int next_chunk(const ProbState* st, int nprob, int prev, double rtol, int max_cycles) {
  int soonest = std::min(2 * prev, MG_HRING);
  for (int p = 0; p < nprob; ++p) {
    const ProbState& S = st[p];
    if (!S.active) continue;
    const int it = S.iter;  // residual evaluations so far
    int rem = max_cycles + 1 - it;
    const int d = std::min(std::min(it - 1, prev), MG_HRING - 1);
    if (rtol > 0.0 && d >= 4) {
      const double r1 = S.hist[(it - 1) % MG_HRING], r0 = S.hist[(it - 1 - d) % MG_HRING];
      const double rho = (r0 > 0.0 && r1 > 0.0) ? pow(r1 / r0, 1.0 / d) : 1.0;
      if (rho < 0.9999) rem = std::min(rem, (int)std::min(1e6, ceil(log(rtol / r1) / log(rho))) + 1);
    }
    soonest = std::min(soonest, std::max(rem, 1));
  }
  const int G = (soonest + kGraphCycles - 1) / kGraphCycles * kGraphCycles;
  return std::min(std::max(G, kGraphCycles), MG_HRING / kGraphCycles * kGraphCycles);
}

// row pitch of level vectors: a multiple of 32 floats (128-byte rows, TMA-aligned)
static int pitch_of(int n) { return (n + 31) & ~31; }

// Workspace layout; with base == nullptr only the size is computed.  Level vectors are
// level-major: r and e of all problems of a level form one pitched [nprob][n][pitch]
// array, the unit of the TMA tensor maps.
static size_t carve(const Plan& P, const mg_options& o, void* base, mg_ctx* ctx) {
  Carver c(base);
  ProbDev* probs = c.take<ProbDev>(P.nprob);
  ProbState* state = c.take<ProbState>(P.nprob);
  float* partials = c.take<float>((size_t)P.nprob * P.ntiles_max);
  float* xlo = c.take<float>((size_t)P.nprob * P.n0 * P.n0);
  int* fail_flag = c.take<int>(4);
  int* active = c.take<int>(P.nprob);
  NetJob* jobs = c.take<NetJob>((size_t)P.nprob * P.L);
  // scratch for the transposition of one problem's level-0 kernels (smoother_transpose)
  float* tscr = (o.smoother_transpose && (P.hk == HK_FIELD || P.hk == HK_STACK3))
                    ? c.take<float>((size_t)(P.hk == HK_STACK3 ? 27 : 9) * P.n0 * P.n0)
                    : nullptr;
  // the linear smoother: its weights per level (shared by all problems) and three scratch
  // vectors of level-0 size for the chain and the up-sweep residual
  const int lin_lev = P.L > 1 ? P.L - 1 : 1, lin_groups = o.net_per_problem ? P.nprob : 1;
  float* lin = P.hk == HK_LINEAR ? c.take<float>((size_t)MG_NPARAMS_LIN * lin_lev * lin_groups) : nullptr;
  // the shared-kernel network's parameter sets expanded to the dense layout
  const bool shared_net = (P.hk == HK_TABLE || P.hk == HK_FIELD) && o.net_arch == MG_NET_CONV_SHARED;
  float* net_dense = shared_net ? c.take<float>((size_t)MG_NPARAMS * (o.net_levels > 1 ? o.net_levels : 1)) : nullptr;
  float* lin_s[3] = {nullptr, nullptr, nullptr};
  if (P.generic)
    for (int k = 0; k < 3; ++k) lin_s[k] = c.take<float>((size_t)P.nprob * P.n0 * pitch_of(P.n0));
  LevelArrays A;
  memset(&A, 0, sizeof(A));
  for (int l = 0; l < P.L; ++l) {
    A.n[l] = P.nl[l];
    A.pitch[l] = pitch_of(P.nl[l]);
    const size_t sz = (size_t)P.nprob * A.n[l] * A.pitch[l];
    A.r[l] = c.take<float>(sz);
    A.e[l] = c.take<float>(sz);
    // tiled levels >= 1 of either coarse-level layout (the layout of the workspace does not
    // depend on which one the device can run)
    if (l >= 1 && l < P.lstar1) A.f[l] = c.take<float>(sz);
  }
  if (P.lstar1 > 0) {
    const size_t sz = (size_t)P.nprob * A.n[0] * A.pitch[0];
    A.xh0 = c.take<float>(sz);
    A.xl0 = c.take<float>(sz);
    A.b0 = c.take<float>(sz);
    A.r0b = c.take<float>(sz);
    A.xh0b = c.take<float>(sz);
    A.xl0b = c.take<float>(sz);
  }
  std::vector<ProbDev> hp(ctx ? P.nprob : 0);
  for (int p = 0; p < P.nprob; ++p) {
    ProbDev d;
    memset(&d, 0, sizeof(d));
    for (int l = 0; l < P.L; ++l) {
      const int n = P.nl[l];
      const size_t nn = (size_t)n * n;
      LevelDev& v = d.lv[l];
      v.n = n;
      v.T = n < MG_PROXY ? n : MG_PROXY;
      v.pitch = A.pitch[l];
      v.r = A.r[l] ? A.r[l] + (size_t)p * n * A.pitch[l] : nullptr;
      v.e = A.e[l] ? A.e[l] + (size_t)p * n * A.pitch[l] : nullptr;
      v.f = (l >= 1 && l < P.lstar && A.f[l]) ? A.f[l] + (size_t)p * n * A.pitch[l] : v.e;
      if (P.sk == SK_FIELD) v.st = c.take<float>(9 * nn);
      if (l < P.L - 1) {
        if (P.hk == HK_FIELD) v.W = c.take<float>(9 * nn);
        else if (P.hk == HK_TABLE) v.W = c.take<float>((size_t)9 * v.T * v.T);
        else if (P.hk == HK_LINEAR) v.W = lin + (size_t)MG_NPARAMS_LIN * ((o.net_per_problem ? p * lin_lev : 0) + l);
        else if (P.hk == HK_STACK3) v.W = c.take<float>(27 * nn);
      }
    }
    d.m = P.nl[P.L - 1] * P.nl[P.L - 1];
    d.nu1 = P.nu1;
    d.nu2 = P.nu2;
    d.chol = c.take<double>((size_t)d.m * d.m);
    if (ctx) hp[p] = d;
  }
  if (ctx) {
    ctx->h_probs.swap(hp);
    ctx->args.probs = probs;
    ctx->args.state = state;
    ctx->args.partials = partials;
    ctx->args.xh0 = A.xh0;
    ctx->args.xl0 = A.xl0;
    ctx->args.r0a = A.r[0];
    ctx->args.b0 = A.b0;
    ctx->args.r0b = A.r0b;
    ctx->args.xh0b = A.xh0b;
    ctx->args.xl0b = A.xl0b;
    ctx->arrays = A;
    ctx->xlo_ws = xlo;
    ctx->d_fail = fail_flag;
    ctx->d_jobs = jobs;
    ctx->d_active = active;
    ctx->tscratch = tscr;
    ctx->lin = lin;
    ctx->net_dense = net_dense;
    ctx->args.lin_wa = lin_s[0];
    ctx->args.lin_wb = lin_s[1];
    ctx->args.lin_t = lin_s[2];
  }
  return c.off + 256;
}

static void rotated_stencil(double eps, double theta, double s[9]) {
  // Q1 element stiffness of -div(K grad u), K = [[a, b], [b, c]] (closed form)
  const double cs = cos(theta), sn = sin(theta);
  const double a = cs * cs + eps * sn * sn, c = sn * sn + eps * cs * cs, b = cs * sn * (1.0 - eps);
  const double corner = -(a + c) / 6.0;
  s[0] = corner - b / 2;  s[1] = (a - 2 * c) / 3;  s[2] = corner + b / 2;
  s[3] = (c - 2 * a) / 3; s[4] = 4 * (a + c) / 3;  s[5] = (c - 2 * a) / 3;
  s[6] = corner + b / 2;  s[7] = (a - 2 * c) / 3;  s[8] = corner - b / 2;
}

extern "C" {

mg_status mg_rotated_stencil(double eps, double theta, float out[9]) {
  if (!out || !(eps > 0.0)) return fail(MG_ERR_INVALID_ARG, "mg_rotated_stencil: bad arguments");
  double s[9];
  rotated_stencil(eps, theta, s);
  for (int k = 0; k < 9; ++k) out[k] = (float)s[k];
  return MG_OK;
}

size_t mg_workspace_size(const mg_problem* problems, int nprob, const mg_options* opts) {
  Plan P;
  if (make_plan(problems, nprob, opts, P) != MG_OK) return 0;
  return carve(P, *opts, nullptr, nullptr);
}

int mg_net_nparams(void) { return MG_NPARAMS; }

int mg_net_param_count(int arch) {
  return arch == MG_NET_CONV ? MG_NPARAMS : arch == MG_NET_FC ? MG_NPARAMS_FC : arch == MG_NET_LINEAR ? MG_NPARAMS_LIN
         : arch == MG_NET_CONV3 ? MG_NPARAMS_K3 : arch == MG_NET_CONV_SHARED ? MG_NPARAMS_SHARED : 0;
}

mg_status mg_setup(const mg_problem* problems, int nprob, const mg_options* opts, const float* net_params,
                   void* workspace, size_t ws_bytes, void* stream, mg_ctx** out) {
  if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  Plan P;
  mg_status st = make_plan(problems, nprob, opts, P);
  if (st != MG_OK) return st;
  if (opts->smoother == MG_SMOOTH_CNN && !net_params) return fail(MG_ERR_INVALID_ARG, "CNN smoother needs net_params");
  const size_t need = carve(P, *opts, nullptr, nullptr);
  if (!workspace || ws_bytes < need) return fail(MG_ERR_WORKSPACE, "workspace needs %zu bytes, got %zu", need, ws_bytes);
  if (((uintptr_t)workspace & 255) != 0) return fail(MG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  if (P.ctail && !ctail_supported(P.sk, P.hk, ctail_smem_bytes(P.nl, P.lstar, P.L, P.hk))) {
    P.ctail = 0;  // the device cannot hold the cluster: one CTA per problem below MG_TAIL_N
    P.lstar = P.lstar1;
  }
  mg_ctx* ctx = new mg_ctx();
  ctx->plan = P;
  ctx->opts = *opts;
  carve(P, *opts, workspace, ctx);
  CycleArgs& a = ctx->args;
  a.ntiles_max = P.ntiles_max;
  a.nprob = P.nprob;
  a.n0 = P.n0;
  a.L = P.L;
  a.lstar = P.lstar;
  a.ctail = P.ctail;
  for (int l = 0; l < MG_MAXL; ++l) a.nl[l] = P.nl[l];
  a.sk = P.sk;
  a.hk = P.hk;
  a.omega = opts->omega;
  a.stream = s;
  a.prof = &ctx->prof;
  a.active = nullptr;
  a.nactive = 0;
  a.pdl = false;
  a.maps = &ctx->maps;
  a.arrays = &ctx->arrays;
  // pinned, so that the per-chunk read of the control blocks is asynchronous and several
  // contexts can keep their streams busy at once
  if (cudaMallocHost((void**)&ctx->h_state, sizeof(ProbState) * P.nprob) != cudaSuccess) {
    delete ctx;
    return fail(MG_ERR_CUDA, "cudaMallocHost of %d control blocks failed", P.nprob);
  }
  a.shape = P.shape;
  a.strip_rows = 32;
  if (P.lstar > 0 && !build_tile_maps(ctx->maps, ctx->arrays, P.nprob, P.lstar, P.shape)) {
    delete ctx;
    return fail(MG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the level arrays");
  }
  a.lin_maps = &ctx->lin_maps;
  a.nu1 = P.nu1;
  a.nu2 = P.nu2;
  a.generic = P.generic;
  if (P.generic && P.lstar > 0 && !build_lin_maps(ctx->lin_maps, ctx->arrays, a.lin_t, a.lin_wa, P.nprob, P.lstar)) {
    delete ctx;
    return fail(MG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the linear smoother's arrays");
  }
  // level-0 stencils
  for (int p = 0; p < nprob; ++p) {
    const mg_problem& q = problems[p];
    LevelDev& v = ctx->h_probs[p].lv[0];
    if (q.kind == MG_PROBLEM_ROTATED) {
      double sd[9];
      rotated_stencil(q.eps, q.theta, sd);
      for (int k = 0; k < 9; ++k) v.s[k] = (float)sd[k];
    } else if (q.kind == MG_PROBLEM_STENCIL) {
      for (int k = 0; k < 9; ++k) v.s[k] = q.data[k];
    }
    if (P.sk == SK_CONST && !(v.s[4] > 0.f)) {
      delete ctx;
      return fail(MG_ERR_INVALID_ARG, "problem %d: stencil diagonal must be positive", p);
    }
  }
  mg_status rc = MG_OK;
  auto run = [&]() -> mg_status {
    CK(cudaMemcpyAsync(a.probs, ctx->h_probs.data(), sizeof(ProbDev) * P.nprob, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->d_fail, 0, sizeof(int), s));
    if (P.sk == SK_FIELD) {
      const size_t nn = (size_t)P.n0 * P.n0;
      for (int p = 0; p < nprob; ++p) {
        float* f0 = ctx->h_probs[p].lv[0].st;
        if (problems[p].kind == MG_PROBLEM_VARCOEF5) CK(launch_varcoef5(P.n0, 1, problems[p].data, 0, f0, 0, s));
        else CK(cudaMemcpyAsync(f0, problems[p].data, 9 * nn * sizeof(float), cudaMemcpyDeviceToDevice, s));
      }
      for (int l = 0; l + 1 < P.L; ++l) CK(launch_rap_field(a.probs, P.nprob, l, P.nl[l + 1], s));
    } else {
      CK(launch_rap_const(a.probs, P.nprob, P.L, s));
    }
    CK(launch_coarsest_factor(a.probs, P.nprob, P.L, P.sk, ctx->d_fail, s));
    if (P.hk == HK_LINEAR && P.L > 1) {
      // the network is the chain itself: level l takes parameter set min(l, net_levels - 1)
      // of the context's group, or of its problem's group with net_per_problem
      const int nsets = opts->net_levels > 1 ? opts->net_levels : 1, groups = opts->net_per_problem ? P.nprob : 1;
      for (int g = 0; g < groups; ++g)
        for (int l = 0; l + 1 < P.L; ++l) {
          const int set = l < nsets ? l : nsets - 1;
          CK(cudaMemcpyAsync(ctx->lin + (size_t)MG_NPARAMS_LIN * ((size_t)g * (P.L - 1) + l),
                             net_params + (size_t)MG_NPARAMS_LIN * ((size_t)g * nsets + set),
                             MG_NPARAMS_LIN * sizeof(float), cudaMemcpyDeviceToDevice, s));
        }
      if (opts->smoother_transpose) CK(launch_transpose_linear(ctx->lin, groups * (P.L - 1), s));
    } else if (P.hk == HK_STACK3 && P.L > 1) {
      // the three-kernel network on every point of every smoothed level (constant stencils
      // included: its kernel fields are per point, not per boundary class)
      std::vector<NetJob> jobs;
      int nm = 0;
      for (int l = 0; l + 1 < P.L; ++l)
        for (int p = 0; p < nprob; ++p) {
          const LevelDev& v = ctx->h_probs[p].lv[l];
          NetJob J;
          J.st = P.sk == SK_FIELD ? v.st : nullptr;
          J.s = P.sk == SK_CONST ? &a.probs[p].lv[l].s[0] : nullptr;  // device address
          J.W = v.W;
          J.n = v.n;
          J.pad_ = 0;
          nm = J.n > nm ? J.n : nm;
          jobs.push_back(J);
        }
      const int nsets = opts->net_levels > 1 ? opts->net_levels : 1;
      if ((size_t)jobs.size() > (size_t)P.nprob * P.L) return fail(MG_ERR_INVALID_ARG, "too many network jobs");
      CK(cudaMemcpyAsync(ctx->d_jobs, jobs.data(), sizeof(NetJob) * jobs.size(), cudaMemcpyHostToDevice, s));
      for (int l = 0; l + 1 < P.L; ++l) {
        const int set = l < nsets ? l : nsets - 1;
        CK(launch_net_forward3(ctx->d_jobs + (size_t)l * nprob, nprob, P.nl[l], net_params + (size_t)set * MG_NPARAMS_K3,
                               opts->omega, s));
      }
      if (opts->smoother_transpose)  // H^T = K1^T K2^T K3^T on every level
        for (int p = 0; p < nprob; ++p)
          for (int l = 0; l + 1 < P.L; ++l) CK(launch_transpose_stack(ctx->h_probs[p].lv[l].W, P.nl[l], ctx->tscratch, s));
      CK(cudaStreamSynchronize(s));  // the host vector must outlive the asynchronous copy
    } else if (P.hk != HK_JACOBI && P.L > 1) {
      // jobs level-major, so that every level can take its own parameter set
      std::vector<NetJob> jobs;
      std::vector<int> first(P.L, 0), nmax(P.L, 0);
      for (int l = 0; l + 1 < P.L; ++l) {
        first[l] = (int)jobs.size();
        for (int p = 0; p < nprob; ++p) {
          const LevelDev& v = ctx->h_probs[p].lv[l];
          NetJob J;
          J.st = P.sk == SK_FIELD ? v.st : nullptr;
          J.s = P.sk == SK_CONST ? &a.probs[p].lv[l].s[0] : nullptr;  // device address
          J.W = v.W;
          J.n = P.sk == SK_FIELD ? v.n : v.T;
          J.pad_ = 0;
          nmax[l] = J.n > nmax[l] ? J.n : nmax[l];
          jobs.push_back(J);
        }
      }
      CK(cudaMemcpyAsync(ctx->d_jobs, jobs.data(), sizeof(NetJob) * jobs.size(), cudaMemcpyHostToDevice, s));
      const bool fc = opts->net_arch == MG_NET_FC;
      const size_t np_set = fc ? MG_NPARAMS_FC : MG_NPARAMS;
      const float* prm_sets = net_params;
      if (ctx->net_dense) {  // MG_NET_CONV_SHARED: expand every set, then the dense network
        CK(launch_net_expand_shared(net_params, ctx->net_dense, opts->net_levels > 1 ? opts->net_levels : 1, s));
        prm_sets = ctx->net_dense;
      }
      auto net = [&](const NetJob* jobs_dev, int njobs, int nm, const float* prm) {
        // the fully connected network's bfloat16 mode runs its GEMMs on the tensor cores
        if (fc && opts->conv_bf16) return launch_fc_forward_tc(jobs_dev, njobs, nm, prm, opts->omega, s);
        return fc ? launch_fc_forward(jobs_dev, njobs, nm, prm, opts->omega, opts->conv_bf16, s)
                  : launch_net_forward(jobs_dev, njobs, nm, prm, opts->omega, opts->conv_bf16, s);
      };
      if (opts->net_levels <= 1) {
        int nm = 0;
        for (int l = 0; l + 1 < P.L; ++l) nm = nmax[l] > nm ? nmax[l] : nm;
        CK(net(ctx->d_jobs, (int)jobs.size(), nm, prm_sets));
      } else {
        for (int l = 0; l + 1 < P.L; ++l) {
          const int set = l < opts->net_levels ? l : opts->net_levels - 1;
          CK(net(ctx->d_jobs + first[l], nprob, nmax[l], prm_sets + (size_t)set * np_set));
        }
      }
      if (opts->smoother_transpose)
        for (int p = 0; p < nprob; ++p)
          for (int l = 0; l + 1 < P.L; ++l) CK(launch_transpose_kernels(ctx->h_probs[p].lv[l].W, P.nl[l], ctx->tscratch, s));
      // the host vector must outlive the asynchronous copy
      CK(cudaStreamSynchronize(s));
    }
    int failed = 0;
    CK(cudaMemcpyAsync(&failed, ctx->d_fail, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (failed) return fail(MG_ERR_NUMERIC, "coarsest operator is not positive definite");
    return MG_OK;
  };
  rc = run();
  if (rc != MG_OK) {
    delete ctx;
    return rc;
  }
  *out = ctx;
  return MG_OK;
}

void mg_destroy(mg_ctx* ctx) { delete ctx; }

int mg_num_levels(const mg_ctx* ctx) { return ctx ? ctx->plan.L : 0; }

int mg_level_n(const mg_ctx* ctx, int level) {
  if (!ctx || level < 0 || level >= ctx->plan.L) return 0;
  return ctx->plan.nl[level];
}

mg_status mg_get_stencil(const mg_ctx* ctx, int prob, int level, float* out, void* stream) {
  if (!ctx || !out || prob < 0 || prob >= ctx->plan.nprob || level < 0 || level >= ctx->plan.L)
    return fail(MG_ERR_INVALID_ARG, "mg_get_stencil: bad arguments");
  CK(launch_expand_stencil(ctx->args.probs, prob, level, ctx->plan.nl[level], ctx->plan.sk, out, (cudaStream_t)stream));
  return MG_OK;
}

mg_status mg_get_kernels(const mg_ctx* ctx, int prob, int level, float* out, void* stream) {
  if (!ctx || !out || prob < 0 || prob >= ctx->plan.nprob || level < 0 || level >= ctx->plan.L - 1)
    return fail(MG_ERR_INVALID_ARG, "mg_get_kernels: bad arguments (smoothed levels are 0..L-2)");
  if (ctx->plan.hk == HK_LINEAR || ctx->plan.hk == HK_STACK3)
    return fail(MG_ERR_UNSUPPORTED, "mg_get_kernels: the smoother is a chain of convolutions, not one 3x3 kernel per point");
  CK(launch_expand_kernels(ctx->args.probs, prob, level, ctx->plan.nl[level], ctx->plan.sk, ctx->plan.hk,
                           ctx->opts.omega, out, (cudaStream_t)stream));
  return MG_OK;
}

mg_status mg_smoother_apply(mg_ctx* ctx, int prob, int level, const float* f, float* u, int nsteps, void* stream) {
  if (!ctx || !f || !u || prob < 0 || prob >= ctx->plan.nprob || level < 0 || level >= ctx->plan.L - 1 || nsteps < 0)
    return fail(MG_ERR_INVALID_ARG, "mg_smoother_apply: bad arguments (smoothed levels are 0..L-2)");
  if (ctx->plan.hk == HK_STACK3)
    return fail(MG_ERR_UNSUPPORTED, "mg_smoother_apply: not implemented for the three-kernel network");
  CycleArgs a = ctx->args;
  a.stream = (cudaStream_t)stream;
  CK(launch_smoother(a, prob, level, f, u, nsteps));
  return MG_OK;
}

mg_status mg_vcycle(mg_ctx* ctx, const float* b, float* x_hi, float* x_lo, float* rel_res, void* stream) {
  if (!ctx || !b || !x_hi) return fail(MG_ERR_INVALID_ARG, "mg_vcycle: ctx, b and x_hi are required");
  CycleArgs a = ctx->args;
  a.stream = (cudaStream_t)stream;
  const int big = 1 << 30;
  CK(cudaMemsetAsync(a.state, 0, sizeof(ProbState) * a.nprob, a.stream));
  CK(launch_bnorm(a, b));
  if (ctx->plan.tail_solve) {
    CK(launch_tail_solve(a, b, x_hi, x_lo, -1.f, big, 1, 1));
  } else {
    const LevelArrays& A = ctx->arrays;
    CK(launch_pack(b, A.b0, A.n[0], A.pitch[0], a.nprob, a.stream));
    CK(launch_pack(x_hi, A.xh0, A.n[0], A.pitch[0], a.nprob, a.stream));
    CK(launch_pack(x_lo, A.xl0, A.n[0], A.pitch[0], a.nprob, a.stream));
    CK(launch_residual(a, -1.f, big));
    CK(launch_cycle(a, -1.f, big, 0));  // ends with the residual of the new iterate
    CK(launch_unpack(A.xh0, A.xh0b, a.state, x_hi, A.n[0], A.pitch[0], a.nprob, a.stream));
    if (x_lo) CK(launch_unpack(A.xl0, A.xl0b, a.state, x_lo, A.n[0], A.pitch[0], a.nprob, a.stream));
  }
  if (rel_res) CK(launch_copy_rel(a.state, rel_res, a.nprob, a.stream));
  return MG_OK;
}

}  // extern "C"

// ------------------------------------------------------------ solve loop
// One context's solve, split so that several contexts can interleave their chunks.
struct SolveRun {
  mg_ctx* ctx = nullptr;
  CycleArgs a;
  const float* b = nullptr;
  float *x_hi = nullptr, *x_lo = nullptr, *xlo = nullptr;
  double rtol = 0.0;
  int max_cycles = 0;
  double* hist = nullptr;
  int* cycles = nullptr;
  std::vector<int> seen;
  int G = kGraphCycles;
  bool done = false;
};

// copies into the pitched arrays, reset of the control blocks, ||b||, initial residual
static mg_status run_begin(SolveRun& R, mg_ctx* ctx, const float* b, float* x_hi, float* x_lo, double rtol,
                           int max_cycles, double* hist, int* cycles, cudaStream_t stream) {
  if (!ctx || !b || !x_hi) return fail(MG_ERR_INVALID_ARG, "mg_solve: ctx, b and x_hi are required");
  if (max_cycles < 0 || max_cycles > 100000000) return fail(MG_ERR_INVALID_ARG, "max_cycles out of range");
  R.ctx = ctx;
  R.a = ctx->args;
  R.a.stream = stream;
  R.b = b;
  R.x_hi = x_hi;
  R.x_lo = x_lo;
  R.xlo = x_lo;
  R.rtol = rtol;
  R.max_cycles = max_cycles;
  R.hist = hist;
  R.cycles = cycles;
  const Plan& P = ctx->plan;
  CycleArgs& a = R.a;
  const LevelArrays& A = ctx->arrays;
  R.seen.assign(P.nprob, 0);
  if (P.tail_solve) {
    if (!R.xlo) {
      R.xlo = ctx->xlo_ws;
      CK(cudaMemsetAsync(R.xlo, 0, sizeof(float) * (size_t)P.nprob * P.n0 * P.n0, a.stream));
    }
  } else {
    // the tiled path iterates on pitched copies (TMA-aligned rows) and copies x back at the end
    CK(launch_pack(b, A.b0, A.n[0], A.pitch[0], a.nprob, a.stream));
    CK(launch_pack(x_hi, A.xh0, A.n[0], A.pitch[0], a.nprob, a.stream));
    CK(launch_pack(x_lo, A.xl0, A.n[0], A.pitch[0], a.nprob, a.stream));
  }
  CK(cudaMemsetAsync(a.state, 0, sizeof(ProbState) * a.nprob, a.stream));
  CK(launch_bnorm(a, b));
  // residual and stopping test of the initial iterate; every cycle ends with those of the new one
  if (!P.tail_solve) CK(launch_residual(a, (float)rtol, max_cycles));
  return MG_OK;
}

// the next chunk of cycles and the asynchronous read of the control blocks
static mg_status run_launch(SolveRun& R) {
  mg_ctx* ctx = R.ctx;
  const Plan& P = ctx->plan;
  CycleArgs& a = R.a;
  const float frtol = (float)R.rtol;
  if (P.tail_solve) {
    CK(launch_tail_solve(a, R.b, R.x_hi, R.xlo, frtol, R.max_cycles, R.G, 0));
  } else if (ctx->prof.on) {  // event timing needs individual launches
    for (int c = 0; c < R.G; ++c) CK(launch_cycle(a, frtol, R.max_cycles, c & 1));
  } else {
    cudaGraphExec_t exec;
    long long nodes = 0;
    mg_status gs = cycle_graph(ctx, a, frtol, R.max_cycles, &exec, &nodes);
    if (gs != MG_OK) return gs;
    for (int c = 0; c < R.G; c += kGraphCycles) CK(cudaGraphLaunch(exec, a.stream));
    ctx->prof.launches += nodes * (R.G / kGraphCycles);
  }
  CK(cudaMemcpyAsync(ctx->h_state, a.state, sizeof(ProbState) * P.nprob, cudaMemcpyDeviceToHost, a.stream));
  return MG_OK;
}

// after the stream has been synchronised: history, compaction, next chunk length
static mg_status run_collect(SolveRun& R) {
  mg_ctx* ctx = R.ctx;
  const Plan& P = ctx->plan;
  CycleArgs& a = R.a;
  ctx->prof.collect();
  int active = 0;
  ctx->h_active.clear();
  for (int p = 0; p < P.nprob; ++p) {
    const ProbState& S = ctx->h_state[p];
    if (R.hist)
      for (int k = R.seen[p]; k < S.iter; ++k) R.hist[(size_t)p * (R.max_cycles + 1) + k] = S.hist[k % MG_HRING];
    R.seen[p] = S.iter;
    active += S.active;
    if (S.active) ctx->h_active.push_back(p);
  }
  if (!active) {
    R.done = true;
    return MG_OK;
  }
  // later chunks launch CTAs only for the problems still iterating
  if (active < a.nprob && active != a.nactive) {
    CK(cudaMemcpyAsync(ctx->d_active, ctx->h_active.data(), sizeof(int) * active, cudaMemcpyHostToDevice, a.stream));
    a.active = ctx->d_active;
    a.nactive = active;
  }
  R.G = next_chunk(ctx->h_state, P.nprob, R.G, R.rtol, R.max_cycles);
  return MG_OK;
}

// copies x back, waits, and maps the problems' final states to a status
static mg_status run_end(SolveRun& R) {
  mg_ctx* ctx = R.ctx;
  const Plan& P = ctx->plan;
  CycleArgs& a = R.a;
  const LevelArrays& A = ctx->arrays;
  if (!P.tail_solve) {
    CK(launch_unpack(A.xh0, A.xh0b, a.state, R.x_hi, A.n[0], A.pitch[0], a.nprob, a.stream));
    if (R.x_lo) CK(launch_unpack(A.xl0, A.xl0b, a.state, R.x_lo, A.n[0], A.pitch[0], a.nprob, a.stream));
    CK(cudaStreamSynchronize(a.stream));
  }
  mg_status rc = MG_OK;
  for (int p = 0; p < P.nprob; ++p) {
    const ProbState& S = ctx->h_state[p];
    if (R.cycles) R.cycles[p] = S.cycles;
    if (S.status == 4) rc = MG_ERR_TIMEOUT;
    else if (S.status == 3 && rc != MG_ERR_TIMEOUT) rc = MG_ERR_NUMERIC;
    else if (S.status == 2 && rc == MG_OK) rc = MG_ERR_NOT_CONVERGED;
  }
  if (rc == MG_ERR_TIMEOUT) fail(rc, "a bounded wait for tile copies expired");
  else if (rc == MG_ERR_NUMERIC) fail(rc, "non-finite residual");
  else if (rc == MG_ERR_NOT_CONVERGED) fail(rc, "max_cycles reached before rtol");
  return rc;
}

// the cycle arguments of a context whose whole hierarchy runs in one CTA per problem
// (for the training step's coarse V-cycle); false for other contexts
void mg::ctx_args(const mg_ctx* ctx, mg::CycleArgs* a) { *a = ctx->args; }

bool mg::ctx_tail_args(const mg_ctx* ctx, mg::CycleArgs* a) {
  if (!ctx || !ctx->plan.tail_solve) return false;
  *a = ctx->args;
  return true;
}

extern "C" {

mg_status mg_solve(mg_ctx* ctx, const float* b, float* x_hi, float* x_lo, double rtol, int max_cycles, double* hist,
                   int* cycles, void* stream) {
  SolveRun R;
  mg_status st = run_begin(R, ctx, b, x_hi, x_lo, rtol, max_cycles, hist, cycles, (cudaStream_t)stream);
  if (st != MG_OK) return st;
  while (!R.done) {
    if ((st = run_launch(R)) != MG_OK) return st;
    CK(cudaStreamSynchronize(R.a.stream));
    if ((st = run_collect(R)) != MG_OK) return st;
  }
  return run_end(R);
}

mg_status mg_solve_multi(mg_ctx* const* ctxs, int nctx, const float* const* b, float* const* x_hi,
                         float* const* x_lo, double rtol, int max_cycles, int* const* cycles, void* const* streams) {
  if (!ctxs || nctx <= 0 || !b || !x_hi) return fail(MG_ERR_INVALID_ARG, "mg_solve_multi: contexts and arrays required");
  for (int k = 0; k < nctx; ++k)
    for (int q = 0; q < k; ++q)
      if (ctxs[k] == ctxs[q]) return fail(MG_ERR_INVALID_ARG, "mg_solve_multi: context %d appears twice", k);
  std::vector<SolveRun> runs(nctx);
  for (int k = 0; k < nctx; ++k) {
    mg_status st = run_begin(runs[k], ctxs[k], b[k], x_hi[k], x_lo ? x_lo[k] : nullptr, rtol, max_cycles, nullptr,
                             cycles ? cycles[k] : nullptr, streams ? (cudaStream_t)streams[k] : nullptr);
    if (st != MG_OK) return st;
  }
  // each context's next chunk goes out as soon as its previous one has been collected, so
  // no stream waits for the slowest context
  auto abort_all = [&](mg_status st) {
    for (SolveRun& R : runs) cudaStreamSynchronize(R.a.stream);
    return st;
  };
  int pending = 0;
  for (SolveRun& R : runs) {
    mg_status st = run_launch(R);
    if (st != MG_OK) return abort_all(st);
    ++pending;
  }
  while (pending) {
    bool progressed = false;
    for (SolveRun& R : runs) {
      if (R.done) continue;
      const cudaError_t q = cudaStreamQuery(R.a.stream);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return abort_all(fail(MG_ERR_CUDA, "mg_solve_multi: %s", cudaGetErrorString(q)));
      progressed = true;
      mg_status st = run_collect(R);
      if (st == MG_OK && !R.done) st = run_launch(R);
      if (st != MG_OK) return abort_all(st);
      if (R.done) --pending;
    }
    if (!progressed) std::this_thread::yield();
  }
  mg_status rc = MG_OK;
  for (SolveRun& R : runs) {
    const mg_status st = run_end(R);
    if (rc == MG_OK) rc = st;
  }
  return rc;
}

mg_status mg_net_fc_forward(int n, int nprob, const float* fields, const float* params, float omega, int bf16,
                            float* W, void* stream) {
  if (n < 1 || n > 8191 || nprob < 1 || nprob > 65535 || !fields || !params || !W)
    return fail(MG_ERR_INVALID_ARG, "mg_net_fc_forward: bad arguments");
  NetBatch B;
  B.st = fields;
  B.W = W;
  B.stride = 9 * (size_t)n * n;
  B.n = n;
  B.pad_ = 0;
  if (bf16) CK(launch_fc_forward_batch_tc(B, nprob, params, omega, (cudaStream_t)stream));
  else CK(launch_fc_forward_batch(B, nprob, params, omega, bf16, (cudaStream_t)stream));
  return MG_OK;
}

mg_status mg_net_forward(int n, int nprob, const float* fields, const float* params, float omega, int conv_bf16,
                         float* W, void* stream) {
  if (n < 1 || n > 8191 || nprob < 1 || nprob > 65535 || !fields || !params || !W)
    return fail(MG_ERR_INVALID_ARG, "mg_net_forward: bad arguments");
  NetBatch B;
  B.st = fields;
  B.W = W;
  B.stride = (size_t)9 * n * n;
  B.n = n;
  B.pad_ = 0;
  CK(launch_net_forward_batch(B, nprob, params, omega, conv_bf16, (cudaStream_t)stream));
  return MG_OK;
}

mg_status mg_solve_times(const mg_ctx* ctx, unsigned long long* start_ns, unsigned long long* done_ns) {
  if (!ctx || !start_ns || !done_ns) return fail(MG_ERR_INVALID_ARG, "mg_solve_times: bad arguments");
  for (int p = 0; p < ctx->plan.nprob; ++p) {
    start_ns[p] = ctx->h_state[p].t_start;
    done_ns[p] = ctx->h_state[p].status != 0 ? ctx->h_state[p].t_done : 0ull;
  }
  return MG_OK;
}

mg_status mg_debug_short_wait(mg_ctx* ctx, int on) {
  if (!ctx) return fail(MG_ERR_INVALID_ARG, "mg_debug_short_wait: ctx is NULL");
  ctx->args.short_wait = on != 0;
  return MG_OK;
}

mg_status mg_debug_strip_rows(mg_ctx* ctx, int rows) {
  if (!ctx) return fail(MG_ERR_INVALID_ARG, "mg_debug_strip_rows: ctx is NULL");
  if (rows < 0) return fail(MG_ERR_INVALID_ARG, "mg_debug_strip_rows: rows %d < 0", rows);
  ctx->args.strip_rows = rows;
  return MG_OK;
}

mg_status mg_profile_enable(mg_ctx* ctx, int enable) {
  if (!ctx) return fail(MG_ERR_INVALID_ARG, "mg_profile_enable: ctx is NULL");
  ctx->prof.reset();
  ctx->prof.on = enable != 0;
  return MG_OK;
}

mg_status mg_profile_read(mg_ctx* ctx, int kernel_class, double* total_ms, long long* launches) {
  if (!ctx || kernel_class < -1 || kernel_class >= PK_NCLASS)
    return fail(MG_ERR_INVALID_ARG, "mg_profile_read: bad arguments");
  ctx->prof.collect();
  if (kernel_class == -1) {
    if (launches) *launches = ctx->prof.launches;
    if (total_ms) *total_ms = 0.0;
    return MG_OK;
  }
  if (total_ms) *total_ms = ctx->prof.ms[kernel_class];
  if (launches) *launches = ctx->prof.count[kernel_class];
  return MG_OK;
}

const char* mg_status_string(mg_status s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_WORKSPACE: return "workspace too small or misaligned";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_NOT_CONVERGED: return "not converged";
    case MG_ERR_NUMERIC: return "numerical failure";
    case MG_ERR_TIMEOUT: return "timeout";
    case MG_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* mg_last_error(void) { return g_err; }

}  // extern "C"
