// Coarse-level kernels (levels >= 1): one thread per (unit, row).
// Coarse levels have few units, so the one-thread-per-unit kernels of the
// fine level leave most of the GPU idle and walk whole block rows
// serially; here floor(32/B) units share a warp, lane r of a unit owns row
// r, blocks are stored column-major per unit ([c*B + r]) so the lanes of a
// unit read consecutive entries, and the rows of a unit's residual are
// exchanged with warp shuffles for the block-inverse and P^T products
// (through shared memory for B = 64, RowWide below).
#pragma once
#include <type_traits>

#include "kernels.cuh"

namespace aggmg {

// Threads per block of the row-lane kernels. 64 (twice the blocks on the
// small levels, e.g. 144 instead of 72 on the 1,024-unit level of the 512^2
// square) measured 0.4% fewer time-steps/s there and 0.3% on the shell.
#ifndef AGG_RL_NT
#define AGG_RL_NT 128
#endif
constexpr int RL_NT = AGG_RL_NT;

template <typename T>
struct CsrBlocks {           // block CSR with column-major blocks
  const int32_t* rowptr;     // [n + 1]
  const int32_t* cols;       // [nnzb]
  const T* vals;             // [nnzb][B*B], entry (r, c) at c*B + r
  int64_t n;
};

template <int B>
struct RowLane {
  static constexpr int UPW = 32 / B;          // units per warp
  int64_t unit;
  int r, base, lane;
  bool active;
  __device__ __forceinline__ RowLane(int64_t n) {
    lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * RL_NT + threadIdx.x) >> 5;
    const int sub = lane / B;
    r = lane - sub * B;
    base = sub * B;
    unit = warp * UPW + sub;
    active = (sub < UPW) && (unit < n);
  }
  // the same for an explicit warp index (persistent kernels loop over warps)
  __device__ __forceinline__ RowLane(int64_t n, int64_t warp) {
    lane = threadIdx.x & 31;
    const int sub = lane / B;
    r = lane - sub * B;
    base = sub * B;
    unit = warp * UPW + sub;
    active = (sub < UPW) && (unit < n);
  }
};

// Coarse levels of B = 64 (Q3 hexahedra): one thread per (unit, row) as
// well, B / 32 warps per unit and RL_NT / B units per block; the rows of a
// unit are exchanged through shared memory (block barrier) instead of warp
// shuffles. One thread per unit walking its 64 x 64 blocks serially left
// these levels latency bound (about 1 ms per step whatever their size).
template <int B>
struct RowWide {
  static_assert(B % 32 == 0 && RL_NT % B == 0, "wide row-lane units are whole warps of a block");
  int64_t unit;
  int r, base;
  bool active;
  __device__ __forceinline__ RowWide(int64_t n) {
    r = threadIdx.x % B;
    base = threadIdx.x - r;
    unit = (int64_t)blockIdx.x * (RL_NT / B) + threadIdx.x / B;
    active = unit < n;
  }
};
template <int B>
using RowOf = typename std::conditional<(B <= 32), RowLane<B>, RowWide<B>>::type;
// shared exchange slots of a row-lane kernel (none for B <= 32)
template <int B>
constexpr int kRowXchg = (B <= 32) ? 1 : RL_NT;

// (A x)_r of the lane's unit. Two ways to overlap the per-block chain of
// loads (column id, then the neighbour's values) measured no faster on
// GB300: ids loaded together and broadcast by warp shuffles (16.6 against
// 11.8 us per level-1 Chebyshev step), and groups of 2-4 blocks loaded
// unconditionally before use (V-cycle 598-603 against 596 us in 2D, 3.3-4.3
// against 3.1 ms on the shell).
template <typename T, int B, typename Ln>
__device__ __forceinline__ T rl_row(const CsrBlocks<T>& A, const Ln& L, const T* __restrict__ x) {
  T s = T(0);
  if (!L.active) return s;
  const int j0 = A.rowptr[L.unit], j1 = A.rowptr[L.unit + 1];
  for (int j = j0; j < j1; ++j) {
    const int col = A.cols[j];
    const T* blk = A.vals + (size_t)j * B * B + L.r;
    const T* xb = x + (size_t)col * B;
#pragma unroll
    for (int c = 0; c < B; ++c) s += blk[c * B] * xb[c];
  }
  return s;
}

// Makes every row value t of the thread's unit readable as row(c): warp
// shuffles for B <= 32; for B = 64 the block's threads store t in xsh and
// meet at a barrier (every thread of the block calls this).
template <typename T, int B>
struct RowValues {
  const RowOf<B>& L;
  T t;
  const T* xsh;
  __device__ __forceinline__ RowValues(const RowOf<B>& L_, T t_, T* xsh_) : L(L_), t(t_), xsh(xsh_) {
    if constexpr (B > 32) {
      xsh_[threadIdx.x] = t_;
      __syncthreads();
    }
  }
  __device__ __forceinline__ T operator()(int c) const {
    if constexpr (B <= 32) return __shfl_sync(0xffffffffu, t, L.base + c);
    else return xsh[L.base + c];
  }
};

// sum_c M[r][c] t_c with t distributed over the unit's lanes (column-major M)
template <typename T, typename TD, int B>
__device__ __forceinline__ T rl_block(const TD* __restrict__ M, const RowOf<B>& L, T t, T* xsh) {
  T s = T(0);
  const TD* m = M + (size_t)L.unit * B * B + L.r;
  const RowValues<T, B> tv(L, t, xsh);
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const T tc = tv(c);
    if (L.active) s += (T)m[c * B] * tc;
  }
  return s;
}

// KIND 0/1/2 as k_cheb, one (unit, row) per thread
template <typename T, typename TD, int B, int KIND>
static __global__ void __launch_bounds__(RL_NT) k_rl_cheb(CsrBlocks<T> A, const TD* __restrict__ Dinv,
                                                          const T* __restrict__ rhs, const T* __restrict__ x_old,
                                                          T* __restrict__ x_new, T* __restrict__ d, T c1, T c2,
                                                          const CGState* st) {
  if (st && st->done) return;
  __shared__ T xsh[kRowXchg<B>];
  const RowOf<B> L(A.n);
  const size_t o = (size_t)L.unit * B + L.r;
  T t = T(0);
  if constexpr (KIND == 0) {
    if (L.active) t = rhs[o];
  } else {
    const T ax = rl_row<T, B>(A, L, x_old);
    if (L.active) t = rhs[o] - ax;
  }
  const T s = rl_block<T, TD, B>(Dinv, L, t, xsh);
  if (!L.active) return;
  const T dn = (KIND == 2) ? c1 * d[o] + c2 * s : c2 * s;
  d[o] = dn;
  x_new[o] = (KIND == 0) ? dn : x_old[o] + dn;
}

// KIND 0 on a level whose right-hand side is still spread over the finer
// level's restriction sums: rhs_K[r] = sum over the children u of K of
// S_u[r] (children contiguous, summed in k_segsum's order, so the result is
// bitwise that of k_segsum followed by KIND 0), stored for the later steps;
// then d = c2 Dinv rhs, x_new = d.
template <typename T, typename TD, int B>
static __global__ void __launch_bounds__(RL_NT)
    k_rl_cheb_restricted(CsrBlocks<T> A, const TD* __restrict__ Dinv, const int64_t* __restrict__ child_ptr,
                         const T* __restrict__ S, T* __restrict__ rhs, T* __restrict__ x_new, T* __restrict__ d, T c2,
                         const CGState* st) {
  if (st && st->done) return;
  __shared__ T xsh[kRowXchg<B>];
  const RowOf<B> L(A.n);
  const size_t o = (size_t)L.unit * B + L.r;
  T t = T(0);
  if (L.active) {
#pragma unroll 4
    for (int64_t u = child_ptr[L.unit]; u < child_ptr[L.unit + 1]; ++u) t += S[(size_t)u * B + L.r];
    rhs[o] = t;
  }
  const T s = rl_block<T, TD, B>(Dinv, L, t, xsh);
  if (!L.active) return;
  const T dn = c2 * s;
  d[o] = dn;
  x_new[o] = dn;
}

// S_u[j] = sum_i P_u[i][j] (rhs - A x)_u[i]   (P column-major: (i, j) at j*B + i)
template <typename T, int B>
static __global__ void __launch_bounds__(RL_NT) k_rl_resid_restrict(CsrBlocks<T> A, const T* __restrict__ P,
                                                                    const T* __restrict__ rhs, const T* __restrict__ x,
                                                                    T* __restrict__ S, const CGState* st) {
  if (st && st->done) return;
  __shared__ T xsh[kRowXchg<B>];
  const RowOf<B> L(A.n);
  const size_t o = (size_t)L.unit * B + L.r;
  T t = T(0);
  const T ax = rl_row<T, B>(A, L, x);
  if (L.active) t = rhs[o] - ax;
  // lane j (as column index) needs P[i][j] for all i: entries j*B + i, i.e. row j of P^T
  T s = T(0);
  const T* pj = P + (size_t)L.unit * B * B + (size_t)L.r * B;
  const RowValues<T, B> tv(L, t, xsh);
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const T ti = tv(i);
    if (L.active) s += pj[i] * ti;
  }
  if (L.active) S[o] = s;
}

// x_u[r] += sum_j P_u[r][j] e_parent[j]
template <typename T, int B>
static __global__ void __launch_bounds__(RL_NT) k_rl_prolong(const T* __restrict__ P, const int32_t* __restrict__ parent,
                                                             const T* __restrict__ ec, T* __restrict__ x, int64_t n,
                                                             const CGState* st) {
  if (st && st->done) return;
  const RowOf<B> L(n);
  if (!L.active) return;
  const T* pr = P + (size_t)L.unit * B * B + L.r;
  const T* eb = ec + (size_t)parent[L.unit] * B;
  T s = T(0);
#pragma unroll
  for (int j = 0; j < B; ++j) s += pr[j * B] * eb[j];
  x[(size_t)L.unit * B + L.r] += s;
}

// y = A x (levels >= 1, for agg_operator_apply)
template <typename T, int B>
static __global__ void __launch_bounds__(RL_NT) k_rl_spmv(CsrBlocks<T> A, const T* __restrict__ x, T* __restrict__ y) {
  const RowOf<B> L(A.n);
  const T s = rl_row<T, B>(A, L, x);
  if (L.active) y[(size_t)L.unit * B + L.r] = s;
}

template <int B>
inline int64_t rl_grid(int64_t n) {
  if constexpr (B > 32) {
    return (n + RL_NT / B - 1) / (RL_NT / B);
  } else {
    const int64_t warps = (n + RowLane<B>::UPW - 1) / RowLane<B>::UPW;
    return (warps * 32 + RL_NT - 1) / RL_NT;
  }
}

}  // namespace aggmg
