// Persistent kernel for the coarse part of the V-cycle (Section 6): every
// level l >= 1 with its Chebyshev block-Jacobi steps, residual restriction,
// segmented sums, prolongation, and the coarsest level's Cholesky solve, in
// one launch. Coarse levels are small (16K..64 units on the 2D benchmark
// workload), so as separate kernels they cost about 20 launches of a few
// microseconds each per V-cycle, mostly launch latency and idle tails; here
// the phases are separated by grid-wide barriers instead.
//
// Each phase does, per (unit, row) or per coarsest row, exactly the
// arithmetic of the corresponding separate kernel (k_rl_cheb,
// k_rl_resid_restrict, k_segsum, k_rl_prolong, k_coarse_lower/upper) in the
// same order, so both paths give bitwise the same correction.
//
// Measured on GB300 (512^2 Q2 workload, float32 V-cycle): a grid barrier
// costs 2.7-3.9 us (152-608 blocks) while consecutive kernels of a CUDA
// graph start 0.7 us apart, so this kernel (653 us per V-cycle) loses to the
// separate kernels (597 us); it is an option (agg_mg_opts.coarse_persistent),
// not the default.
//
// The launch is cooperative (all blocks resident). Every barrier spins a
// bounded number of times: if the limit is reached the kernel records an
// error, marks the solve done with status AGG_ECUDA and every block leaves
// at its next barrier, so a failure ends the solve instead of hanging it.
//
// Vectors written by one phase and read by a later one are read with
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
  PLevel<T, TD> lev[PMAXL];       // lev[l] for l = 1 .. nl (the smoothed coarse levels)
  int nl;                         // number of smoothed coarse levels (L - 2)
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
  int j0 = 0, len = 0;
  if (L.active) {
    j0 = __ldg(A.rowptr + L.unit);
    len = __ldg(A.rowptr + L.unit + 1) - j0;
  }
  const int wmax = __reduce_max_sync(0xffffffffu, len);
  for (int jb = 0; jb < wmax; jb += B) {
    const int colv = (jb + L.r < len) ? __ldg(A.cols + j0 + jb + L.r) : -1;
#pragma unroll
    for (int jj = 0; jj < B; ++jj) {
      const int col = __shfl_sync(0xffffffffu, colv, (L.base + jj) & 31);
      if (L.active && col >= 0) {
        const T* blk = A.vals + (size_t)(j0 + jb + jj) * B * B + L.r;
        const T* xb = x + (size_t)col * B;
#pragma unroll
        for (int c = 0; c < B; ++c) s += __ldg(blk + c * B) * __ldcg(xb + c);
      }
    }
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
    const T ax = p_row<T, B>(v.A, L, x_old);      // every lane (warp shuffles)
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
  const T ax = p_row<T, B>(v.A, L, x);            // every lane (warp shuffles)
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
  for (int64_t k = row + lane; k < n; k += 32) s += __ldg(Ur + k) * __ldcg(y + k);
  s = warp_sum(s);
  if (lane == 0) z[row] = (T)s;
}

// Warps needed by a row-lane phase on n units.
template <int B>
__device__ __forceinline__ int64_t rl_warps(int64_t n) {
  return (n + RowLane<B>::UPW - 1) / RowLane<B>::UPW;
}

template <typename T, typename TD, int B>
static __global__ void __launch_bounds__(PNT, 5) k_coarse_persistent(PCoarse<T, TD> P) {
  if (P.st->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * PNT + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * PNT) >> 5;
  const int64_t gthr = (int64_t)blockIdx.x * PNT + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * PNT;
  T* xo[PMAXL + 1];
  T* xn[PMAXL + 1];
  bool ok = true;
#define AGG_PHASE_END                   \
  if (!(ok = grid_sync(P.bar, P.extra))) goto fail;
  // ---- down: pre-smoothing, residual, restriction
  for (int l = 1; l <= P.nl; ++l) {
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
  for (int l = P.nl; l >= 1; --l) {
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

}  // namespace aggmg
