// mg_krylov.cu -- flexible GMRES with the multigrid V-cycle as the preconditioner
// (Sec. 6.4), batched over the problems of a context.
//
// Right preconditioning: z_j = M v_j with M one V(1,1) cycle from zero of the context (its
// smoother, Jacobi or network), w = A z_j, classical Gram-Schmidt with one
// re-orthogonalisation against v_0 .. v_j, v_{j+1} = w / ||w||.  The small Hessenberg
// problem (Givens rotations, the triangular solve) is solved on the host per problem;
// every vector operation runs on the device over all problems at once.  The preconditioner
// is "flexible": the stored z_j, not M, enter x = x0 + Z y, so a preconditioner that is not
// a fixed linear map is allowed.
//
// The iterate is float-float, x = x_hi + x_lo: at 511^2 the rounding of an FP32 iterate
// alone leaves a relative residual near 1e-5, above the 1e-6 the experiments ask for.  So
// every restart (and the final check) evaluates b - A x with the compensated Dot2
// product, and x += Z y is added with an error-free sum; the Krylov vectors are FP32.
// Inner products are summed in float-float in a fixed order (deterministic): per-CTA
// partial sums of a fixed chunk of the vector, then the chunks in order.
#include <math.h>
#include <string.h>

#include <vector>

#include "mg_internal.h"
#include "mgcnn.h"

namespace mg {

constexpr int KT = 256;      // threads per CTA of the vector kernels
constexpr int KCHUNK = 32;   // CTAs (chunks) per vector of an inner product

// y_p = A_p x_p on level 0, dense [nprob][n][n] vectors
template <int SK>
__global__ void k_kry_applyA(const ProbDev* __restrict__ probs, const float* __restrict__ x, float* __restrict__ y,
                             const float* __restrict__ b) {
  const int p = blockIdx.y;
  const LevelDev& L = probs[p].lv[0];
  const int n = L.n;
  const size_t nn = (size_t)n * n;
  const int q = blockIdx.x * KT + threadIdx.x;
  if (q >= (int)nn) return;
  const int i = q / n, j = q % n;
  const float* xp = x + (size_t)p * nn;
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
    if (!in_grid(ii, jj, n)) continue;
    const float a = (SK == SK_CONST) ? L.s[k] : __ldg(L.st + k * nn + q);
    acc = fmaf(a, xp[ii * n + jj], acc);
  }
  // b given: the residual b - A x
  y[(size_t)p * nn + q] = b ? b[(size_t)p * nn + q] - acc : acc;
}

// r_p = b_p - A_p (xh_p + xl_p), Dot2: exact products and error-free sums for xh, FP32
// for the xl terms (the x_lo part is below an ulp of x_hi)
template <int SK>
__global__ void k_kry_residual(const ProbDev* __restrict__ probs, const float* __restrict__ b,
                               const float* __restrict__ xh, const float* __restrict__ xl, float* __restrict__ r) {
  const int p = blockIdx.y;
  const LevelDev& L = probs[p].lv[0];
  const int n = L.n;
  const size_t nn = (size_t)n * n;
  const int q = blockIdx.x * KT + threadIdx.x;
  if (q >= (int)nn) return;
  const int i = q / n, j = q % n;
  const float* xhp = xh + (size_t)p * nn;
  const float* xlp = xl + (size_t)p * nn;
  float hi = b[(size_t)p * nn + q], lo = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ii = i + k / 3 - 1, jj = j + k % 3 - 1;
    if (!in_grid(ii, jj, n)) continue;
    const float a = (SK == SK_CONST) ? L.s[k] : __ldg(L.st + k * nn + q);
    const float x = xhp[ii * n + jj];
    const float pr = __fmul_rn(a, x), pe = fmaf(a, x, -pr);
    float sum, err;
    two_sum(hi, -pr, sum, err);
    hi = sum;
    lo = __fadd_rn(lo, __fsub_rn(err, pe));
    lo = fmaf(-a, xlp[ii * n + jj], lo);
  }
  r[(size_t)p * nn + q] = __fadd_rn(hi, lo);
}

// (xh, xl) += sum_i coef[p * nv + i] Z_i,p  (the sum in FP32, added error-free)
__global__ void k_kry_update(float* __restrict__ xh, float* __restrict__ xl, const float* __restrict__ Z,
                             size_t vstride, size_t nn, int nv, const float* __restrict__ coef) {
  const int p = blockIdx.y;
  const size_t q = (size_t)blockIdx.x * KT + threadIdx.x;
  if (q >= nn) return;
  float acc = 0.f;
  for (int i = 0; i < nv; ++i) acc = fmaf(coef[(size_t)p * nv + i], Z[i * vstride + (size_t)p * nn + q], acc);
  const size_t o = (size_t)p * nn + q;
  float s, e;
  two_sum(xh[o], acc, s, e);
  e = __fadd_rn(e, xl[o]);
  fast_two_sum(s, e, xh[o], xl[o]);
}

// partial inner products: part[((p * nv + i) * KCHUNK) + c] = <V_i,p , w_p> over chunk c
__global__ void k_kry_dots(const float* __restrict__ V, size_t vstride, const float* __restrict__ w, size_t nn,
                           int nv, float* __restrict__ part) {
  __shared__ float sh[KT / 32], sl[KT / 32];
  const int c = blockIdx.x, i = blockIdx.y, p = blockIdx.z;
  const size_t len = (nn + KCHUNK - 1) / KCHUNK, a = c * len, e = min(nn, a + len);
  const float* v = V + i * vstride + (size_t)p * nn;
  const float* x = w + (size_t)p * nn;
  float hi = 0.f, lo = 0.f;
  for (size_t q = a + threadIdx.x; q < e; q += KT) {
    const float pr = __fmul_rn(v[q], x[q]);
    ff_add(hi, lo, pr, fmaf(v[q], x[q], -pr));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, oh, ol);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = hi;
    sl[threadIdx.x >> 5] = lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float h = 0.f, l = 0.f;
    for (int k = 0; k < KT / 32; ++k) ff_add(h, l, sh[k], sl[k]);
    part[2 * (((size_t)p * nv + i) * KCHUNK + c)] = h;
    part[2 * (((size_t)p * nv + i) * KCHUNK + c) + 1] = l;
  }
}

// out[p * nv + i] = sum of the chunks in order (double)
__global__ void k_kry_dots_final(const float* __restrict__ part, int count, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double s = 0.0;
  for (int c = 0; c < KCHUNK; ++c) s += (double)part[2 * ((size_t)t * KCHUNK + c)] + (double)part[2 * ((size_t)t * KCHUNK + c) + 1];
  out[t] = s;
}

// w_p += sign * sum_i coef[p * nv + i] V_i,p   (sign -1: Gram-Schmidt; +1: x += Z y)
__global__ void k_kry_axpy(float* __restrict__ w, const float* __restrict__ V, size_t vstride, size_t nn, int nv,
                           const float* __restrict__ coef, float sign) {
  const int p = blockIdx.y;
  const size_t q = (size_t)blockIdx.x * KT + threadIdx.x;
  if (q >= nn) return;
  float acc = 0.f;
  for (int i = 0; i < nv; ++i) acc = fmaf(coef[(size_t)p * nv + i], V[i * vstride + (size_t)p * nn + q], acc);
  w[(size_t)p * nn + q] = fmaf(sign, acc, w[(size_t)p * nn + q]);
}

// out_p = s_p w_p; out and w may be the same array (the restart scales V_0 in place), so
// neither is declared restrict
__global__ void k_kry_scale(float* out, const float* w, size_t nn, const float* __restrict__ s) {
  const int p = blockIdx.y;
  const size_t q = (size_t)blockIdx.x * KT + threadIdx.x;
  if (q >= nn) return;
  out[(size_t)p * nn + q] = s[p] * w[(size_t)p * nn + q];
}

}  // namespace mg

using namespace mg;

namespace {

struct KrylovWs {
  float *V, *Z, *w, *xl, *part, *coef;
  double* dots;
  size_t bytes;
};

KrylovWs kry_carve(int nprob, int n, int m, void* base) {
  KrylovWs k;
  size_t off = 0;
  char* b = (char*)base;
  const size_t nn = (size_t)n * n, vec = nn * nprob;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    void* p = b ? b + off : nullptr;
    off += bytes;
    return p;
  };
  k.V = (float*)take(sizeof(float) * vec * (m + 1));
  k.Z = (float*)take(sizeof(float) * vec * m);
  k.w = (float*)take(sizeof(float) * vec);
  k.xl = (float*)take(sizeof(float) * vec);  // x_lo when the caller passes none
  k.part = (float*)take(sizeof(float) * 2 * (size_t)nprob * (m + 1) * KCHUNK);
  k.coef = (float*)take(sizeof(float) * (size_t)nprob * (m + 1));
  k.dots = (double*)take(sizeof(double) * (size_t)nprob * (m + 1));
  k.bytes = off + 256;
  return k;
}

#define KCK(call)                                                                                       \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return (mg_status)api_fail(MG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" {

size_t mg_fgmres_workspace_size(const mg_ctx* ctx, int restart) {
  if (!ctx || restart < 1 || restart > 200) return 0;
  CycleArgs a;
  ctx_args(ctx, &a);
  return kry_carve(a.nprob, a.n0, restart, nullptr).bytes;
}

mg_status mg_fgmres(mg_ctx* ctx, const float* b, float* x_hi, float* x_lo, int restart, double rtol, int max_iters,
                    void* workspace, size_t ws_bytes, double* hist, int* iters, void* stream) {
  if (!ctx || !b || !x_hi || restart < 1 || restart > 200 || max_iters < 0 || !(rtol > 0.0))
    return (mg_status)api_fail(MG_ERR_INVALID_ARG, "mg_fgmres: bad arguments");
  CycleArgs a;
  ctx_args(ctx, &a);
  const int np = a.nprob, n = a.n0, m = restart;
  const KrylovWs K = kry_carve(np, n, m, workspace);
  if (!workspace || ws_bytes < K.bytes)
    return (mg_status)api_fail(MG_ERR_WORKSPACE, "mg_fgmres workspace needs %zu bytes, got %zu", K.bytes, ws_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nn = (size_t)n * n, vec = nn * np;
  const dim3 gv((unsigned)((nn + KT - 1) / KT), np);
  auto applyA = [&](const float* in, float* out, const float* bb) -> cudaError_t {
    if (a.sk == SK_CONST) k_kry_applyA<SK_CONST><<<gv, KT, 0, s>>>(a.probs, in, out, bb);
    else k_kry_applyA<SK_FIELD><<<gv, KT, 0, s>>>(a.probs, in, out, bb);
    return cudaGetLastError();
  };
  float* xl = x_lo;
  if (!xl) {
    xl = K.xl;
    KCK(cudaMemsetAsync(xl, 0, sizeof(float) * vec, s));
  }
  // compensated r = b - A (x_hi + x_lo)
  auto residual = [&](float* out) -> cudaError_t {
    if (a.sk == SK_CONST) k_kry_residual<SK_CONST><<<gv, KT, 0, s>>>(a.probs, b, x_hi, xl, out);
    else k_kry_residual<SK_FIELD><<<gv, KT, 0, s>>>(a.probs, b, x_hi, xl, out);
    return cudaGetLastError();
  };
  std::vector<double> hd((size_t)np * (m + 1));
  // <V_0..nv-1 (stride vstride), w> for every problem, to the host
  auto dots = [&](const float* Vb, size_t vstride, int nv, const float* w) -> mg_status {
    k_kry_dots<<<dim3(KCHUNK, nv, np), KT, 0, s>>>(Vb, vstride, w, nn, nv, K.part);
    const int cnt = np * nv;
    k_kry_dots_final<<<(cnt + 127) / 128, 128, 0, s>>>(K.part, cnt, K.dots);
    KCK(cudaGetLastError());
    KCK(cudaMemcpyAsync(hd.data(), K.dots, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    KCK(cudaStreamSynchronize(s));
    return MG_OK;
  };
  std::vector<float> hc((size_t)np * (m + 1));
  auto put_coef = [&](int nv) -> cudaError_t {
    return cudaMemcpyAsync(K.coef, hc.data(), sizeof(float) * np * nv, cudaMemcpyHostToDevice, s);
  };
  // ||b|| per problem
  mg_status st = dots(b, 0, 1, b);
  if (st != MG_OK) return st;
  std::vector<double> bnorm(np);
  for (int p = 0; p < np; ++p) bnorm[p] = sqrt(hd[p]);
  std::vector<int> its(np, 0), done(np, 0);
  std::vector<double> H((size_t)np * (m + 1) * m), g((size_t)np * (m + 1)), cs((size_t)np * m), sn((size_t)np * m);
  std::vector<int> len(np);
  int it = 0;
  for (;;) {
    // r = b - A x into V_0 (compensated), beta = ||r||
    KCK(residual(K.V));
    if ((st = dots(K.V, 0, 1, K.V)) != MG_OK) return st;
    int active = 0;
    for (int p = 0; p < np; ++p) {
      const double beta = sqrt(hd[p]);
      const double rel = bnorm[p] > 0.0 ? beta / bnorm[p] : 0.0;
      if (it == 0 && hist) hist[(size_t)p * (max_iters + 1)] = rel;
      if (!done[p] && (rel < rtol || its[p] >= max_iters || beta == 0.0)) done[p] = 1;
      active += !done[p];
      g[(size_t)p * (m + 1)] = beta;
      hc[p] = (!done[p] && beta > 0.0) ? (float)(1.0 / beta) : 0.f;
      len[p] = done[p] ? 0 : -1;
    }
    if (!active) break;
    KCK(cudaMemcpyAsync(K.coef, hc.data(), sizeof(float) * np, cudaMemcpyHostToDevice, s));
    k_kry_scale<<<gv, KT, 0, s>>>(K.V, K.V, nn, K.coef);
    int j = 0, running = active;
    for (; j < m && running; ++j) {
      float* vj = K.V + j * vec;
      float* zj = K.Z + j * vec;
      KCK(cudaMemsetAsync(zj, 0, sizeof(float) * vec, s));
      st = mg_vcycle(ctx, vj, zj, nullptr, nullptr, s);
      if (st != MG_OK) return st;
      KCK(applyA(zj, K.w, nullptr));
      // two classical Gram-Schmidt passes
      for (int pass = 0; pass < 2; ++pass) {
        if ((st = dots(K.V, vec, j + 1, K.w)) != MG_OK) return st;
        for (int p = 0; p < np; ++p)
          for (int i = 0; i <= j; ++i) {
            const double h = len[p] == -1 ? hd[(size_t)p * (j + 1) + i] : 0.0;
            double& Hij = H[((size_t)p * (m + 1) + i) * m + j];
            Hij = pass == 0 ? h : Hij + h;
            hc[(size_t)p * (j + 1) + i] = (float)h;
          }
        KCK(put_coef(j + 1));
        k_kry_axpy<<<gv, KT, 0, s>>>(K.w, K.V, vec, nn, j + 1, K.coef, -1.f);
      }
      if ((st = dots(K.w, 0, 1, K.w)) != MG_OK) return st;
      for (int p = 0; p < np; ++p) {
        const double hn = sqrt(hd[p]);
        hc[p] = (len[p] == -1 && hn > 0.0) ? (float)(1.0 / hn) : 0.f;
        if (len[p] != -1) continue;
        double* Hp = &H[(size_t)p * (m + 1) * m];
        double* gp = &g[(size_t)p * (m + 1)];
        double* c = &cs[(size_t)p * m];
        double* sv = &sn[(size_t)p * m];
        Hp[(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {  // earlier rotations
          const double t = c[i] * Hp[i * m + j] + sv[i] * Hp[(i + 1) * m + j];
          Hp[(i + 1) * m + j] = -sv[i] * Hp[i * m + j] + c[i] * Hp[(i + 1) * m + j];
          Hp[i * m + j] = t;
        }
        const double rho = hypot(Hp[j * m + j], Hp[(j + 1) * m + j]);
        c[j] = rho > 0.0 ? Hp[j * m + j] / rho : 1.0;
        sv[j] = rho > 0.0 ? Hp[(j + 1) * m + j] / rho : 0.0;
        Hp[j * m + j] = rho;
        Hp[(j + 1) * m + j] = 0.0;
        gp[j + 1] = -sv[j] * gp[j];
        gp[j] = c[j] * gp[j];
        ++its[p];
        const double rel = fabs(gp[j + 1]) / bnorm[p];
        if (hist && its[p] <= max_iters) hist[(size_t)p * (max_iters + 1) + its[p]] = rel;
        if (rel < rtol || its[p] >= max_iters || hn == 0.0) {
          len[p] = j + 1;
          --running;
        }
      }
      KCK(cudaMemcpyAsync(K.coef, hc.data(), sizeof(float) * np, cudaMemcpyHostToDevice, s));
      k_kry_scale<<<gv, KT, 0, s>>>(K.V + (j + 1) * vec, K.w, nn, K.coef);
    }
    // x += Z y, y from the triangular system of each problem's own length
    for (int p = 0; p < np; ++p) {
      int lp = len[p] == -1 ? j : len[p];
      if (done[p]) lp = 0;
      const double* Hp = &H[(size_t)p * (m + 1) * m];
      const double* gp = &g[(size_t)p * (m + 1)];
      std::vector<double> y(lp);
      for (int r = lp - 1; r >= 0; --r) {
        double acc = gp[r];
        for (int c2 = r + 1; c2 < lp; ++c2) acc -= Hp[r * m + c2] * y[c2];
        y[r] = acc / Hp[r * m + r];
      }
      for (int i = 0; i < j; ++i) hc[(size_t)p * j + i] = i < lp ? (float)y[i] : 0.f;
    }
    if (j > 0) {
      KCK(put_coef(j));
      k_kry_update<<<gv, KT, 0, s>>>(x_hi, xl, K.Z, vec, nn, j, K.coef);
      KCK(cudaGetLastError());
    }
    it += j;
  }
  // the true (compensated) residual decides the status
  KCK(residual(K.w));
  if ((st = dots(K.w, 0, 1, K.w)) != MG_OK) return st;
  int rc = MG_OK;
  for (int p = 0; p < np; ++p) {
    if (iters) iters[p] = its[p];
    if (bnorm[p] > 0.0 && sqrt(hd[p]) / bnorm[p] >= rtol) rc = MG_ERR_NOT_CONVERGED;
  }
  if (rc != MG_OK) api_fail(rc, "mg_fgmres: max_iters reached before rtol");
  return (mg_status)rc;
}

}  // extern "C"
