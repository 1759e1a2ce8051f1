// mg_ctail.cu -- the coarse levels of the V-cycle (Algorithm 1) in one thread-block
// cluster per problem, for sm_103a.
//
// Levels of side n_l <= MG_CT_N(hk, n_0) run in a cluster of MG_CT_C CTAs per problem, every
// vector in shared memory.  On a band level (n_l > MG_CT_SOLO(hk, n_0)) CTA k owns the rows
// [k B, k B + B), B = (n_l + 1) / MG_CT_C (the last CTA one row fewer), and keeps r, e and
// t of its band with MG_CT_HD halo rows on each side, a zero column on each side and zero
// rows outside the grid (the Dirichlet exterior).  Levels of side <= MG_CT_SOLO(hk, n_0) run in
// CTA 0 alone on whole ring-padded arrays, down to the FP64 coarsest solve and back.
//
// Down step of a band level: e = H r on the band and two halo rows, t = r - A e on the
// band and one halo row, then r_c = P^T t on the CTA's coarse rows.  Only r_c crosses CTAs:
// its first and last MG_CT_HD rows are also stored into the neighbours' halo rows through
// distributed shared memory (into CTA 0's whole array when the coarse level is solo), and
// the cluster synchronises once.  Up step: e += P e_c on the band and two halo rows,
// t = r - A e on the band and one, e_final = e + H t on the band; the rows of e_final a
// neighbour's prolongation needs (the first row for the CTA above, the last two for the
// CTA below) go to a separate array, because the neighbour still reads its own halo rows
// of e while they are sent.  Cluster barriers per cycle: one after the prologue, one per
// band level on the way down, one after the solo levels, one per band level on the way up
// below the top.
#include <atomic>

#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_ops.cuh"
#include "mg_tail.cuh"
#include "mg_tma.cuh"

namespace mg {

// threads per CTA of the cluster tail: 512 lets two CTAs share an SM, so the clusters of a
// 16-problem batch and more are resident at once (with 1024 threads at most 14 clusters of
// eight CTAs fit on the GPU and a 16-problem tail ran in two waves)
#ifndef MG_CT_THREADS
#define MG_CT_THREADS 512
#endif
constexpr int CT_THREADS = MG_CT_THREADS;
// A band of the smallest band level (side 2 MG_CT_SOLO + 1) must hold the MG_CT_HD rows it
// pushes into each neighbour's halo.
static_assert((2 * MG_CT_SOLO_SHORT + 2) / MG_CT_C >= MG_CT_HD && (2 * MG_CT_SOLO_LONG + 2) / MG_CT_C >= MG_CT_HD,
              "band levels need at least MG_CT_HD rows per CTA");

struct CtLayout {
  TailLayout a;         // r, e, t (band or whole arrays) and kernel tables of every level
  int off_p[MG_MAXL];   // band levels below the top: final e as the finer prolongation reads it
  int band[MG_MAXL];    // rows per CTA on band levels, 0 on solo levels
  int lsolo;            // first solo level
};

__host__ __device__ inline void ct_layout(const int* nl, int ls, int L, int hk, CtLayout& t) {
  int lsolo = ls;
  while (lsolo < L && nl[lsolo] > MG_CT_SOLO(hk, nl[0])) ++lsolo;
  t.lsolo = lsolo;
  int o = 0;
  for (int l = ls; l < L; ++l) {
    const int m = nl[l] + 2;
    int sz;
    if (l < lsolo) {
      t.band[l] = (nl[l] + 1) / MG_CT_C;
      sz = (t.band[l] + 2 * MG_CT_HD) * m;
    } else {
      t.band[l] = 0;
      sz = m * m;
    }
    t.a.off_r[l] = o; o += sz;
    t.a.off_e[l] = o; o += sz;
    t.a.off_t[l] = o; o += sz;
    t.off_p[l] = -1;
    if (l > ls && l < lsolo) { t.off_p[l] = o; o += sz; }
  }
  tail_layout_tables(nl, ls, L, hk, o, t.a);
}

// ------------------------------------------------------------- cluster PTX
__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}

// Every thread of every CTA of the cluster; shared-memory stores before it, local or
// remote, are visible to every thread of the cluster after it.  The non-.aligned form
// counts threads one by one, so lanes need not have reconverged after a divergent loop.
__device__ __forceinline__ void cluster_sync() {
  asm volatile(
      "barrier.cluster.arrive.release;\n\t"
      "barrier.cluster.wait.acquire;" ::: "memory");
}

// generic address of the same shared-memory location in CTA `rank` of the cluster
template <class T>
__device__ __forceinline__ T* cluster_map(T* p, int rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
  return reinterpret_cast<T*>(out);
}

// rows [a, b) of a level of side n: work items of one row and 32 columns spread over warps
// (n + 1 is a power of two, so is the number of 32-column chunks per row: shifts, no division)
#define CT_FOR(a, b, n)                                                                                \
  for (int it_ = warp, sh_ = 31 - __clz(((n) + 31) >> 5), end_ = ((b) - (a)) << sh_; it_ < end_;        \
       it_ += nwarps)                                                                                  \
    for (int i = (a) + (it_ >> sh_), j = ((it_ & ((1 << sh_) - 1)) << 5) + lane; j < (n); j = (n))

// Zero columns, rows outside the grid and solo-level rings; stencil constants, class
// tables, interior kernels and the coarsest inverse of levels ls .. L-1.  Ends with a
// barrier.
template <int SK, int HK>
__device__ void ct_prologue(const ProbDev& P, float* sm, const CtLayout& lay, float (*sc)[9], float (*wi)[9], int ls,
                            int L, int rank) {
  load_level_data<SK, HK>(P, sm, lay.a, sc, ls, L);
  for (int l = ls; l < L; ++l) {
    const int n = lay.a.n[l], m = n + 2;
    const int offs[4] = {lay.a.off_r[l], lay.a.off_e[l], lay.a.off_t[l], lay.off_p[l]};
    if (l < lay.lsolo) {
      const int B = lay.band[l], R = B + 2 * MG_CT_HD, i0 = rank * B;
      const int za = i0 < MG_CT_HD ? MG_CT_HD - i0 : 0;  // local rows [0, za) lie above row 0
      const int zb = n + MG_CT_HD - i0;                  // local rows [zb, R) lie below row n-1
      for (int a = 0; a < 4; ++a) {
        if (offs[a] < 0) continue;
        float* v = sm + offs[a];
        for (int k = threadIdx.x; k < R; k += blockDim.x) {
          v[k * m] = 0.f;
          v[k * m + m - 1] = 0.f;
        }
        for (int k = threadIdx.x; k < za * m; k += blockDim.x) v[k] = 0.f;
        if (zb < R)
          for (int k = zb * m + threadIdx.x; k < R * m; k += blockDim.x) v[k] = 0.f;
      }
    } else if (rank == 0) {
      for (int a = 0; a < 3; ++a) {
        float* v = sm + offs[a];
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
          v[k] = 0.f;
          v[(m - 1) * m + k] = 0.f;
          v[k * m] = 0.f;
          v[k * m + m - 1] = 0.f;
        }
      }
    }
  }
  __syncthreads();
  load_interior_kernels<HK>(sm, lay.a, wi, ls, L);
  __syncthreads();
}

// Down step of band level l (pre-smoothing from e = 0, residual, restriction).
template <int SK, int HK>
__device__ void ct_down(const ProbDev& P, float* sm, const CtLayout& lay, const float (*sc)[9],
                        const float (*wi)[9], int l, int rank, float omega) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const LevelDev& V = P.lv[l];
  const int n = lay.a.n[l], m = n + 2, B = lay.band[l], i0 = rank * B, i1 = min(i0 + B, n);
  const int o = MG_CT_HD - i0;  // local row of grid row i: i + o
  const float* r = sm + lay.a.off_r[l];
  float* e = sm + lay.a.off_e[l];
  float* t = sm + lay.a.off_t[l];
  const float* w = sm + lay.a.off_w[l];
  float sr[9], wr[9];  // stencil and interior kernel in registers
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    sr[k] = sc[l][k];
    wr[k] = wi[l][k];
  }
  CT_FOR(max(0, i0 - 2), min(n, i1 + 2), n) {
    const int q = (i + o) * m + j + 1;
    e[q] = pad_H<SK, HK>(V, sr, w, wr, omega, r + q, m, n, i, j);
  }
  __syncthreads();
  CT_FOR(max(0, i0 - 1), min(n, i1 + 1), n) {
    const int q = (i + o) * m + j + 1;
    t[q] = r[q] - pad_A<SK>(V, sr, e + q, m, n, i, j);
  }
  __syncthreads();
  // coarse rows [I0, I1) of this CTA: fine rows 2I .. 2I+2 lie in the band and its first
  // lower halo row
  const int nc = lay.a.n[l + 1], mc = nc + 2, Bc = B >> 1, I0 = rank * Bc, I1 = min(I0 + Bc, nc);
  float* rc = sm + lay.a.off_r[l + 1];
  if (l + 1 < lay.lsolo) {
    float* up = rank > 0 ? cluster_map(rc, rank - 1) : nullptr;
    float* dn = rank < MG_CT_C - 1 ? cluster_map(rc, rank + 1) : nullptr;
    const int oc = MG_CT_HD - I0;
    CT_FOR(I0, I1, nc) {
      const float v = restrict_at(t + (2 * i + 1 + o) * m + 2 * j + 2, m);
      const int q = (i + oc) * mc + j + 1;
      rc[q] = v;
      if (up && i < I0 + MG_CT_HD) up[q + Bc * mc] = v;   // lower halo of the CTA above
      if (dn && i >= I1 - MG_CT_HD) dn[q - Bc * mc] = v;  // upper halo of the CTA below
    }
  } else {
    if (rank != 0) rc = cluster_map(rc, 0);
    CT_FOR(I0, I1, nc) rc[(i + 1) * mc + j + 1] = restrict_at(t + (2 * i + 1 + o) * m + 2 * j + 2, m);
  }
  cluster_sync();
}

// Up step of band level l (prolongation and correction, residual, post-smoothing); the
// top level ls writes its final e to the pitched level array.
template <int SK, int HK>
__device__ void ct_up(const ProbDev& P, float* sm, const CtLayout& lay, const float (*sc)[9], const float (*wi)[9],
                      int l, int ls, int rank, float omega) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const LevelDev& V = P.lv[l];
  const int n = lay.a.n[l], m = n + 2, B = lay.band[l], i0 = rank * B, i1 = min(i0 + B, n);
  const int o = MG_CT_HD - i0;
  const float* r = sm + lay.a.off_r[l];
  float* e = sm + lay.a.off_e[l];
  float* t = sm + lay.a.off_t[l];
  const float* w = sm + lay.a.off_w[l];
  const int mc = lay.a.n[l + 1] + 2;
  const bool solo_below = l + 1 == lay.lsolo;
  const float* ec;
  int Io;  // coarse grid row of the first stored row of ec
  if (!solo_below) {
    ec = sm + lay.off_p[l + 1];
    Io = rank * (B >> 1) - MG_CT_HD;
  } else {
    float* e0 = sm + lay.a.off_e[l + 1];
    ec = rank == 0 ? e0 : cluster_map(e0, 0);
    Io = -1;
  }
  float sr[9], wr[9];  // stencil and interior kernel in registers
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    sr[k] = sc[l][k];
    wr[k] = wi[l][k];
  }
  CT_FOR(max(0, i0 - 2), min(n, i1 + 2), n) e[(i + o) * m + j + 1] += prolong_at(i, j, ec, Io, -1, mc);
  __syncthreads();
  CT_FOR(max(0, i0 - 1), min(n, i1 + 1), n) {
    const int q = (i + o) * m + j + 1;
    t[q] = r[q] - pad_A<SK>(V, sr, e + q, m, n, i, j);
  }
  __syncthreads();
  if (l > ls) {
    float* pl = sm + lay.off_p[l];
    float* up = rank > 0 ? cluster_map(pl, rank - 1) : nullptr;
    float* dn = rank < MG_CT_C - 1 ? cluster_map(pl, rank + 1) : nullptr;
    CT_FOR(i0, i1, n) {
      const int q = (i + o) * m + j + 1;
      const float v = e[q] + pad_H<SK, HK>(V, sr, w, wr, omega, t + q, m, n, i, j);
      pl[q] = v;
      if (up && i == i0) up[q + B * m] = v;      // lower halo of the CTA above
      if (dn && i >= i1 - 2) dn[q - B * m] = v;  // upper halo of the CTA below
    }
    cluster_sync();
  } else {
    CT_FOR(i0, i1, n) {
      const int q = (i + o) * m + j + 1;
      V.e[(size_t)i * V.pitch + j] = e[q] + pad_H<SK, HK>(V, sr, w, wr, omega, t + q, m, n, i, j);
    }
    if (solo_below) cluster_sync();  // CTA 0 keeps its arrays until every CTA has read them
  }
}

// One cycle of levels ls .. L-1 for problem act[blockIdx.y]; blockIdx.x is the rank in
// the cluster.  Reads r_ls and writes e_ls (pitched level arrays).
template <int SK, int HK>
__global__ void __launch_bounds__(CT_THREADS, CT_THREADS <= 512 ? 2 : 1) k_ctail(const ProbDev* __restrict__ probs,
                                                         const ProbState* __restrict__ state, int ls, int L,
                                                         float omega, const int* __restrict__ act) {
  extern __shared__ float sm[];
  __shared__ float sc[MG_MAXL][9];
  __shared__ float wi[MG_MAXL][9];
  __shared__ CtLayout lay;
  pdl_trigger();
  const int rank = cluster_rank();
  const int p = act ? act[blockIdx.y] : blockIdx.y;
  const ProbDev& P = probs[p];
  if (threadIdx.x == 0) {
    int nl[MG_MAXL];
    for (int l = 0; l < L; ++l) nl[l] = P.lv[l].n;
    ct_layout(nl, ls, L, HK, lay);
  }
  __syncthreads();
  const float* rtop = P.lv[ls].r;  // before the wait: descriptors do not change
  const int rpitch = P.lv[ls].pitch;
  ct_prologue<SK, HK>(P, sm, lay, sc, wi, ls, L, rank);
  pdl_wait();
  __shared__ int live;
  if (threadIdx.x == 0) live = st_active(state + p);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  {
    const int n = lay.a.n[ls], m = n + 2, i0 = rank * lay.band[ls];
    const int a = max(0, i0 - MG_CT_HD), b = min(n, i0 + lay.band[ls] + MG_CT_HD);
    float* r = sm + lay.a.off_r[ls];
    CT_FOR(a, b, n) r[(i - i0 + MG_CT_HD) * m + j + 1] = __ldcg(rtop + (size_t)i * rpitch + j);
  }
  cluster_sync();  // every CTA of the cluster is running with its exterior zeroed
  // Leave or stay as a whole cluster, on CTA 0's reading of the flag: a CTA that left
  // while the others went on would break their barriers and shared-memory pushes.
  if (!*cluster_map(&live, 0)) {
    cluster_sync();  // CTA 0 keeps `live` until every CTA has read it
    return;
  }
  const int lsolo = lay.lsolo;
  for (int l = ls; l < lsolo; ++l) ct_down<SK, HK>(P, sm, lay, sc, wi, l, rank, omega);
  if (rank == 0) tail_cycle<SK, HK>(P, sm, lay.a, sc, wi, lsolo, L, omega);
  cluster_sync();
  for (int l = lsolo - 1; l >= ls; --l) ct_up<SK, HK>(P, sm, lay, sc, wi, l, ls, rank, omega);
}

// ---------------------------------------------------------------- launchers
size_t ctail_smem_bytes(const int* nl, int ls, int L, int hk) {
  CtLayout lay;
  ct_layout(nl, ls, L, hk, lay);
  return (size_t)lay.a.total * sizeof(float);
}

// raises the dynamic shared-memory limit of the kernel once per device
template <int SK, int HK>
static cudaError_t ctail_attrs() {
  static std::atomic<int> done[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(k_ctail<SK, HK>, cudaFuncAttributeMaxDynamicSharedMemorySize, MG_CT_SMEM_MAX);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev].store(1, std::memory_order_release);
  return e;
}

static cudaLaunchConfig_t ctail_config(dim3 grid, size_t smem, cudaStream_t s, bool pdl, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(CT_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = MG_CT_C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 2 : 1;
  return cfg;
}

bool ctail_supported(int sk, int hk, size_t smem) {
  if (smem > MG_CT_SMEM_MAX) return false;
  cudaError_t e;
  MG_DISPATCH(sk, hk, (e = ctail_attrs<SK_, HK_>()));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchAttribute at[2];
  cudaLaunchConfig_t cfg = ctail_config(dim3(MG_CT_C, 1), smem, 0, false, at);
  int clusters = 0;
  MG_DISPATCH(sk, hk, (e = cudaOccupancyMaxActiveClusters(&clusters, k_ctail<SK_, HK_>, &cfg)));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters > 0;
}

cudaError_t prepare_ctail(const CycleArgs& a) {
  cudaError_t e;
  MG_DISPATCH(a.sk, a.hk, (e = ctail_attrs<SK_, HK_>()));
  return e;
}

cudaError_t launch_ctail(const CycleArgs& a) {
  if (a.hk == HK_LINEAR || a.hk == HK_STACK3) return cudaErrorNotSupported;  // never planned with these smoothers
  const int ls = a.lstar, L = a.L;
  const size_t smem = ctail_smem_bytes(a.nl, ls, L, a.hk);
  cudaError_t e = prepare_ctail(a);
  if (e != cudaSuccess) return e;
  const int np = (a.active && a.nactive > 0) ? a.nactive : a.nprob;
  cudaLaunchAttribute at[2];
  cudaLaunchConfig_t cfg = ctail_config(dim3(MG_CT_C, np), smem, a.stream, a.pdl, at);
  a.prof->launches++;
  a.prof->begin(PK_TAIL, a.stream);
  const ProbDev* probs = a.probs;
  const ProbState* state = a.state;
  const float omega = a.omega;
  const int* act = a.active;
  MG_DISPATCH(a.sk, a.hk, (e = cudaLaunchKernelEx(&cfg, k_ctail<SK_, HK_>, probs, state, ls, L, omega, act)));
  a.prof->end(a.stream);
  return e;
}

}  // namespace mg
