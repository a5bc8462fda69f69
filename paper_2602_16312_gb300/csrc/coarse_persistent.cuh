// Coarse part of the V-cycle (Section 6) in one launch: the levels from a
// first level on, with their Chebyshev block-Jacobi steps, residual
// restriction, segmented sums, prolongation, and the coarsest level's
// Cholesky solve, the steps separated by barriers instead of kernel
// boundaries. Two forms:
//   k_coarse_persistent: levels >= 1 on the whole GPU, cooperative launch,
//     software grid barrier (agg_mg_opts.coarse_persistent);
//   k_coarse_cluster: the smallest levels (each at most 16 x 1024 rows) on
//     one thread-block cluster of 16 (else 8) CTAs, separated by the
//     cluster's hardware barrier (agg_mg_opts.coarse_cluster).
//
// Each step does, per (unit, row) or per coarsest row, exactly the
// arithmetic of the corresponding separate kernel (k_rl_cheb,
// k_rl_resid_restrict, k_segsum, k_rl_prolong, k_coarse_lower/upper) in the
// same order, so all paths give bitwise the same correction.
//
// Measured on GB300 (float32 V-cycle), both are options and not defaults:
//   - a grid barrier costs 2.7-3.9 us (152-608 blocks), while consecutive
//     kernels of a CUDA graph start 0.7 us apart; V-cycle of the 512^2 Q2
//     workload 646-653 us persistent against 593-597 us separate;
//   - the cluster kernel: 593.8 against 595.6 us (512^2 Q2, levels 2-3),
//     3,067 against 3,037 us (64^3 Q2 cube), 3,184 against 3,110 us (shell).
//   The coarse steps are bound by each thread's chain of dependent loads
//   (neighbour column id, then its block values), which fusing launches does
//   not shorten.
//
// The cooperative launch keeps all blocks resident. Every grid barrier spins
// a bounded number of times: if the limit is reached the kernel records an
// error, marks the solve done with status AGG_ECUDA and every block leaves
// at its next barrier, so a failure ends the solve instead of hanging it.
// The cluster barrier is the hardware's; every CTA of the cluster reaches
// each one (the early exit on a finished solve is taken by all of them).
//
// Vectors written by one step and read by a later one are read with
// __ldcg (L2, coherent); operator, block and map data with __ldg.
#pragma once
#include "coarse_kernels.cuh"
#include "kernels.cuh"

namespace aggmg {

constexpr int PNT = 256;              // threads per block of the persistent kernel
constexpr int PMAXL = 16;             // levels (the R*-tree can give deep hierarchies)
constexpr int PMAXDEG = 8;            // Chebyshev degree
constexpr unsigned kBarrierSpins = 1u << 22;   // ~0.3 s at 64 ns per spin

template <typename T, typename TD>
struct PLevel {
  CsrBlocks<T> A;                 // column-major blocks
  const TD* Dinv;                 // column-major B x B per unit
  const T* P;                     // column-major prolongation blocks to the next level
  const int32_t* parent;          // [n] unit of the next level
  const int64_t* child_ptr;       // [n + 1] this level's children on the previous level
  T *rhs, *xa, *xb, *d, *S;
  T c1[PMAXDEG], c2[PMAXDEG];
  int64_t n;
};

template <typename T, typename TD>
struct PCoarse {
  PLevel<T, TD> lev[PMAXL];       // lev[l] for l = first .. nl (the smoothed coarse levels run here)
  int first;                      // first level run here (1 for the grid-wide kernel)
  int nl;                         // last smoothed level (L - 2)
  int degree;
  // coarsest level (index nl + 1)
  int64_t n_c_units;
  const int64_t* child_ptr_c;
  T* rhs_c;
  T* x_c;
  const double* Linv;
  const double* U;
  double* yc;
  int64_t nc;
  GridBar* bar;
  CGState* st;
  // arrivals a barrier waits for beyond the grid's blocks: 0, except in the
  // test of the timeout path, where the extra arrivals never come
  unsigned extra;
};

// Grid barrier; false (in every thread of the block) once any block has
// recorded an error.
__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned extra) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    volatile int* verr = &b->err;
    int good = (*verr == 0);
    if (good) {
      const unsigned g = *vgen;
      __threadfence();
      if (atomicAdd(&b->count, 1u) == gridDim.x + extra - 1) {
        atomicExch(&b->count, 0u);
        __threadfence();
        atomicAdd(&b->gen, 1u);
      } else {
        unsigned it = 0;
        while (*vgen == g) {
          if (*verr) break;
          if (++it > kBarrierSpins) {
            atomicExch(&b->err, 1);
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
      good = (*verr == 0);
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// ---- phase bodies (one item each), same arithmetic as the separate kernels

template <typename T, int B>
__device__ __forceinline__ T p_row(const CsrBlocks<T>& A, const RowLane<B>& L, const T* x) {
  T s = T(0);
  if (!L.active) return s;
  const int j0 = __ldg(A.rowptr + L.unit), j1 = __ldg(A.rowptr + L.unit + 1);
  for (int j = j0; j < j1; ++j) {
    const int col = __ldg(A.cols + j);
    const T* blk = A.vals + (size_t)j * B * B + L.r;
    const T* xb = x + (size_t)col * B;
#pragma unroll
    for (int c = 0; c < B; ++c) s += __ldg(blk + c * B) * __ldcg(xb + c);
  }
  return s;
}

template <typename T, typename TD, int B>
__device__ __forceinline__ T p_block(const TD* M, const RowLane<B>& L, T t) {
  T s = T(0);
  const TD* m = M + (size_t)L.unit * B * B + L.r;
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const T tc = __shfl_sync(0xffffffffu, t, L.base + c);
    if (L.active) s += (T)__ldg(m + c * B) * tc;
  }
  return s;
}

template <typename T, typename TD, int B, int KIND>
__device__ __forceinline__ void p_cheb(const PLevel<T, TD>& v, const T* x_old, T* x_new, T c1, T c2, int64_t warp) {
  const RowLane<B> L(v.A.n, warp);
  const size_t o = (size_t)L.unit * B + L.r;
  T t = T(0);
  if constexpr (KIND == 0) {
    if (L.active) t = __ldcg(v.rhs + o);
  } else {
    const T ax = p_row<T, B>(v.A, L, x_old);
    if (L.active) t = __ldcg(v.rhs + o) - ax;
  }
  const T s = p_block<T, TD, B>(v.Dinv, L, t);
  if (!L.active) return;
  const T dn = (KIND == 2) ? c1 * __ldcg(v.d + o) + c2 * s : c2 * s;
  v.d[o] = dn;
  x_new[o] = (KIND == 0) ? dn : __ldcg(x_old + o) + dn;
}

template <typename T, typename TD, int B>
__device__ __forceinline__ void p_resid_restrict(const PLevel<T, TD>& v, const T* x, int64_t warp) {
  const RowLane<B> L(v.A.n, warp);
  const size_t o = (size_t)L.unit * B + L.r;
  T t = T(0);
  const T ax = p_row<T, B>(v.A, L, x);
  if (L.active) t = __ldcg(v.rhs + o) - ax;
  T s = T(0);
  const T* pj = v.P + (size_t)L.unit * B * B + (size_t)L.r * B;
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const T ti = __shfl_sync(0xffffffffu, t, L.base + i);
    if (L.active) s += __ldg(pj + i) * ti;
  }
  if (L.active) v.S[o] = s;
}

template <typename T, int B>
__device__ __forceinline__ void p_segsum(const int64_t* child_ptr, const T* S, T* rc, int64_t nK, int64_t id) {
  if (id >= nK * B) return;
  const int64_t K = id / B;
  const int j = (int)(id % B);
  T s = T(0);
#pragma unroll 4
  for (int64_t u = __ldg(child_ptr + K); u < __ldg(child_ptr + K + 1); ++u) s += __ldcg(S + (size_t)u * B + j);
  rc[id] = s;
}

template <typename T, typename TD, int B>
__device__ __forceinline__ void p_prolong(const PLevel<T, TD>& v, const T* ec, T* x, int64_t warp) {
  const RowLane<B> L(v.A.n, warp);
  if (!L.active) return;
  const T* pr = v.P + (size_t)L.unit * B * B + L.r;
  const T* eb = ec + (size_t)__ldg(v.parent + L.unit) * B;
  T s = T(0);
#pragma unroll
  for (int j = 0; j < B; ++j) s += __ldg(pr + j * B) * __ldcg(eb + j);
  x[(size_t)L.unit * B + L.r] += s;
}

template <typename T>
__device__ __forceinline__ void p_coarse_lower(const double* Linv, const T* r, double* y, int64_t n, int64_t row,
                                               int lane) {
  if (row >= n) return;
  const double* Lr = Linv + (size_t)row * n;
  double s = 0.0;
#pragma unroll 8
  for (int64_t k = lane; k <= row; k += 32) s += __ldg(Lr + k) * (double)__ldcg(r + k);
  s = warp_sum(s);
  if (lane == 0) y[row] = s;
}

template <typename T>
__device__ __forceinline__ void p_coarse_upper(const double* U, const double* y, T* z, int64_t n, int64_t row,
                                               int lane) {
  if (row >= n) return;
  const double* Ur = U + (size_t)row * n;
  double s = 0.0;
#pragma unroll 8
  for (int64_t k = row + lane; k < n; k += 32) s += __ldg(Ur + k) * __ldcg(y + k);
  s = warp_sum(s);
  if (lane == 0) z[row] = (T)s;
}

// Warps needed by a row-lane phase on n units.
template <int B>
__device__ __forceinline__ int64_t rl_warps(int64_t n) {
  return (n + RowLane<B>::UPW - 1) / RowLane<B>::UPW;
}

// Phase barriers: the software grid barrier of the cooperative kernel, or the
// hardware barrier of a thread-block cluster (barrier.cluster arrive/wait with
// release/acquire semantics at cluster scope).
struct GridSync {
  GridBar* bar;
  unsigned extra;
  __device__ __forceinline__ bool operator()() const { return grid_sync(bar, extra); }
};
struct ClusterSync {
  __device__ __forceinline__ bool operator()() const {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    return true;
  }
};

// The coarse part of one V-cycle from level P.first down to the coarsest and
// back, on all NTH * gridDim.x threads; level P.first's right-hand side is in
// place. Returns after the last post-smoothing step of level P.first.
template <typename T, typename TD, int B, int NTH, typename Sync>
__device__ __forceinline__ void coarse_cycle(const PCoarse<T, TD>& P, Sync sync) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * NTH + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * NTH) >> 5;
  const int64_t gthr = (int64_t)blockIdx.x * NTH + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * NTH;
  T* xo[PMAXL + 1];
  T* xn[PMAXL + 1];
#define AGG_PHASE_END \
  if (!sync()) goto fail;
  // ---- down: pre-smoothing, residual, restriction
  for (int l = P.first; l <= P.nl; ++l) {
    const PLevel<T, TD>& v = P.lev[l];
    xo[l] = v.xa;
    xn[l] = v.xb;
    const int64_t nw = rl_warps<B>(v.n);
    for (int64_t w = gwarp; w < nw; w += nwarp) p_cheb<T, TD, B, 0>(v, nullptr, xo[l], T(0), v.c2[0], w);
    AGG_PHASE_END
    for (int k = 1; k < P.degree; ++k) {
      for (int64_t w = gwarp; w < nw; w += nwarp) p_cheb<T, TD, B, 2>(v, xo[l], xn[l], v.c1[k], v.c2[k], w);
      AGG_PHASE_END
      T* t = xo[l]; xo[l] = xn[l]; xn[l] = t;
    }
    for (int64_t w = gwarp; w < nw; w += nwarp) p_resid_restrict<T, TD, B>(v, xo[l], w);
    AGG_PHASE_END
    const bool next_coarsest = (l == P.nl);
    const int64_t nK = next_coarsest ? P.n_c_units : P.lev[l + 1].n;
    const int64_t* cp = next_coarsest ? P.child_ptr_c : P.lev[l + 1].child_ptr;
    T* rc = next_coarsest ? P.rhs_c : P.lev[l + 1].rhs;
    for (int64_t id = gthr; id < nK * B; id += nthr) p_segsum<T, B>(cp, v.S, rc, nK, id);
    AGG_PHASE_END
  }
  // ---- coarsest: y = L^{-1} r, x = L^{-T} y
  for (int64_t row = gwarp; row < P.nc; row += nwarp) p_coarse_lower<T>(P.Linv, P.rhs_c, P.yc, P.nc, row, lane);
  AGG_PHASE_END
  for (int64_t row = gwarp; row < P.nc; row += nwarp) p_coarse_upper<T>(P.U, P.yc, P.x_c, P.nc, row, lane);
  // ---- up: prolongation and post-smoothing
  for (int l = P.nl; l >= P.first; --l) {
    AGG_PHASE_END
    const PLevel<T, TD>& v = P.lev[l];
    const T* ec = (l == P.nl) ? P.x_c : xo[l + 1];
    const int64_t nw = rl_warps<B>(v.n);
    for (int64_t w = gwarp; w < nw; w += nwarp) p_prolong<T, TD, B>(v, ec, xo[l], w);
    AGG_PHASE_END
    for (int64_t w = gwarp; w < nw; w += nwarp) p_cheb<T, TD, B, 1>(v, xo[l], xn[l], T(0), v.c2[0], w);
    { T* t = xo[l]; xo[l] = xn[l]; xn[l] = t; }
    for (int k = 1; k < P.degree; ++k) {
      AGG_PHASE_END
      for (int64_t w = gwarp; w < nw; w += nwarp) p_cheb<T, TD, B, 2>(v, xo[l], xn[l], v.c1[k], v.c2[k], w);
      T* t = xo[l]; xo[l] = xn[l]; xn[l] = t;
    }
  }
#undef AGG_PHASE_END
  return;
fail:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.st->status = AGG_ECUDA;
    P.st->done = 1;
  }
}

// Levels >= 1 on the whole GPU (cooperative launch, software grid barrier).
template <typename T, typename TD, int B>
static __global__ void __launch_bounds__(PNT, 5) k_coarse_persistent(PCoarse<T, TD> P) {
  if (P.st->done) return;
  coarse_cycle<T, TD, B, PNT>(P, GridSync{P.bar, P.extra});
}

// The smallest levels (from P.first on, each at most CNT x cluster-size
// rows) in one thread-block cluster of up to 16 CTAs: the grid is the
// cluster, phases are separated by the cluster's hardware barrier.
constexpr int CNT = 1024;
template <typename T, typename TD, int B>
static __global__ void __launch_bounds__(CNT, 1) k_coarse_cluster(PCoarse<T, TD> P) {
  if (P.st->done) return;
  coarse_cycle<T, TD, B, CNT>(P, ClusterSync{});
}

}  // namespace aggmg
