// Device kernels of the per-step hot path (sm_103a).
//
// Data layout ("sliced blocks"): units (elements on level 0, agglomerates on
// coarser levels) are grouped in slices of 32; one thread owns one unit and
// computes its B = (p+1)^d outputs in registers. A B x B block of every unit
// of a slice is stored as KP = B*B (rounded up to 16 bytes) values in the
// order [k / VW][lane][k % VW] with k = c*B + r (c column, r row) and
// VW = 16 / sizeof(T): a warp reads 512 contiguous bytes per vector load.
// Block-sparse operators store one such slot per (slice, neighbour slot)
// plus a column index per (slot, lane); rows with fewer blocks than the
// slice maximum are padded with zero blocks pointing at the row itself.
// Vectors are unit-major: entry u*B + i.
//
// Every kernel of a PCG iteration reads the solver's `done` flag first and
// returns at once when the iteration has converged, so extra launches after
// convergence do no work.
#pragma once
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace aggmg {

constexpr int SL = 32;          // units per slice
constexpr int NT = 128;         // threads per block of the unit kernels (B <= 32)
constexpr int RED_BLOCKS = 1216; // fixed grid of the reduction kernels (152 SMs x 8)
constexpr int RED_NT = 256;

// ---------------------------------------------------------------- PCG state
struct CGState {
  double rho, alpha, beta, pq, rr, r0, tol, rtol, atol;
  double rz_old;              // (r_{k+1}, z_k) for the flexible variant
  int iter, done, status, max_it, flexible, use_cond;
  int guard;                  // WHILE-body executions of this solve (hard stop)
  unsigned long long cond;    // cudaGraphConditionalHandle of the WHILE node
  unsigned ticket[4];         // last-block tickets, one per reduction kind
};

// Grid-wide barrier state of the persistent coarse-level kernel: arrival
// count, generation, error flag (set when a barrier times out).
struct GridBar {
  unsigned count;
  unsigned gen;
  int err;
  int pad;
};

// ---------------------------------------------------------------- vector types
template <typename T> struct Vec;
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<__nv_bfloat16> { using type = uint4; static constexpr int W = 8; };

template <typename T, int B> struct Pad {
  static constexpr int VW = Vec<T>::W;
  static constexpr int KP = ((B * B + VW - 1) / VW) * VW;
  static constexpr int NCH = KP / VW;
};

template <typename T> __device__ __forceinline__ void unpack(const typename Vec<T>::type& v, float* out);
template <> __device__ __forceinline__ void unpack<float>(const float4& v, float* o) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <> __device__ __forceinline__ void unpack<__nv_bfloat16>(const uint4& v, float* o) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    float2 f = __bfloat1622float2(h[t]);
    o[2 * t] = f.x;
    o[2 * t + 1] = f.y;
  }
}

// Loads of data that one launch reads exactly once (operator blocks, smoother
// and transfer blocks, quadrature data). On level 0 (ST, the default) they
// carry the streaming (evict-first) cache hint, so that the L2 keeps the
// vectors, which the neighbouring units read again, and the coarse levels'
// data. Coarse-level blocks (ST = false) take the plain read-only path: the
// smaller coarse levels then stay in L2 from one launch to the next.
#ifndef AGG_STREAM_LOADS
#define AGG_STREAM_LOADS 1
#endif
template <bool ST = true, typename V>
__device__ __forceinline__ V ld_once(const V* p) {
  if constexpr (ST && AGG_STREAM_LOADS) return __ldcs(p);
  else return __ldg(p);
}

// Loads chunk `ch` of a sliced block into vals[0..VW) as the accumulation type A.
template <typename TS, typename A> struct ChunkLoad;
template <> struct ChunkLoad<double, double> {
  static constexpr int VW = 2;
  template <bool ST = true>
  __device__ __forceinline__ static void load(const double* base, int ch, int lane, double* v) {
    double2 t = ld_once<ST>(reinterpret_cast<const double2*>(base) + (size_t)ch * SL + lane);
    v[0] = t.x; v[1] = t.y;
  }
};
template <> struct ChunkLoad<float, float> {
  static constexpr int VW = 4;
  template <bool ST = true>
  __device__ __forceinline__ static void load(const float* base, int ch, int lane, float* v) {
    float4 t = ld_once<ST>(reinterpret_cast<const float4*>(base) + (size_t)ch * SL + lane);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
};
template <> struct ChunkLoad<__nv_bfloat16, float> {
  static constexpr int VW = 8;
  template <bool ST = true>
  __device__ __forceinline__ static void load(const __nv_bfloat16* base, int ch, int lane, float* v) {
    uint4 t = ld_once<ST>(reinterpret_cast<const uint4*>(base) + (size_t)ch * SL + lane);
    unpack<__nv_bfloat16>(t, v);
  }
};

// Threads per block of the unit kernels: 128, or 64 for 64-DoF blocks whose
// per-thread vectors are staged in shared memory.
template <int B> struct UnitThreads {
  static constexpr int value = (B > 32) ? 64 : 128;
};

// Whether the kernels of an operator load its blocks, the smoother blocks and
// the transfer blocks with the streaming hint (see ld_once): true for the
// level-0 operators; the coarse-level block-sparse operator specialises it
// to false.
template <typename Op> struct OpStreams {
  static constexpr bool value = true;
};

// Minimum resident blocks per SM asked of the compiler for the kernels that
// evaluate an operator Op: Op::kMinBlocks where Op has it, else 0 (0 leaves
// the register budget to the compiler's own heuristics, as if no minimum
// were given; an explicit 1 lets it take up to 255 registers).
template <typename Op, typename = void> struct OpMinBlocks {
  static constexpr int value = 0;
};
template <typename Op> struct OpMinBlocks<Op, std::void_t<decltype(Op::kMinBlocks)>> {
  static constexpr int value = Op::kMinBlocks;
};

// acc[r] += sum_c M[r][c] x[c*XS] for one sliced block M (storage TS, math
// A). x may be a register array (XS = 1, fully unrolled indices), a global
// pointer (neighbour blocks, read through L1) or a strided shared-memory slot.
template <typename TS, typename A, int B, int XS = 1, bool ST = true>
__device__ __forceinline__ void block_mv(const TS* base, int lane, const A* x, A* acc) {
  constexpr int VW = ChunkLoad<TS, A>::VW;
  constexpr int NCH = (B * B + VW - 1) / VW;
  if constexpr (B > 32) {
    // large blocks: loop over the columns (chunks never straddle a column
    // since VW divides B), rows unrolled, so acc keeps static indices
    static_assert(B % VW == 0, "column-aligned chunks");
#pragma unroll 1
    for (int c = 0; c < B; ++c) {
      const A xc = x[c * XS];
#pragma unroll
      for (int rr = 0; rr < B / VW; ++rr) {
        A v[VW];
        ChunkLoad<TS, A>::template load<ST>(base, c * (B / VW) + rr, lane, v);
#pragma unroll
        for (int t = 0; t < VW; ++t) acc[rr * VW + t] += v[t] * xc;
      }
    }
    return;
  }
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    A v[VW];
    ChunkLoad<TS, A>::template load<ST>(base, ch, lane, v);
#pragma unroll
    for (int t = 0; t < VW; ++t) {
      const int k = ch * VW + t;
      if (k < B * B) acc[k % B] += v[t] * x[(k / B) * XS];
    }
  }
}
// acc[c] += sum_r M[r][c] x[r*XS] (transposed block)
template <typename TS, typename A, int B, int XS = 1, bool ST = true>
__device__ __forceinline__ void block_mtv(const TS* base, int lane, const A* x, A* acc) {
  constexpr int VW = ChunkLoad<TS, A>::VW;
  constexpr int NCH = (B * B + VW - 1) / VW;
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    A v[VW];
    ChunkLoad<TS, A>::template load<ST>(base, ch, lane, v);
#pragma unroll
    for (int t = 0; t < VW; ++t) {
      const int k = ch * VW + t;
      if (k < B * B) acc[k / B] += v[t] * x[(k % B) * XS];
    }
  }
}

// out[c] = sum_r M[r][c] x[r] for large blocks (B > 32): x in registers,
// one output at a time through a pointer
template <typename TS, typename A, int B, bool ST = true>
__device__ __forceinline__ void block_mtv_out(const TS* base, int lane, const A* x, A* out) {
  constexpr int VW = ChunkLoad<TS, A>::VW;
  static_assert(B % VW == 0, "column-aligned chunks");
#pragma unroll 1
  for (int c = 0; c < B; ++c) {
    A s = A(0);
#pragma unroll
    for (int rr = 0; rr < B / VW; ++rr) {
      A v[VW];
      ChunkLoad<TS, A>::template load<ST>(base, c * (B / VW) + rr, lane, v);
#pragma unroll
      for (int t = 0; t < VW; ++t) s += v[t] * x[rr * VW + t];
    }
    out[c] = s;
  }
}

// Symmetric B x B blocks (the smoother's block inverses, B <= 32) keep their
// upper triangle only, column by column: entry (i, j), i <= j, at
// k = j (j + 1) / 2 + i, in the same sliced chunk layout.
template <typename TS, int B> struct SymPad {
  static constexpr int VW = Vec<TS>::W;
  static constexpr int NP = B * (B + 1) / 2;
  static constexpr int KP = ((NP + VW - 1) / VW) * VW;
};
// Storage of the smoother blocks seen by the unit kernels: packed symmetric
// for B <= 32, full for larger blocks (their column loop needs full columns).
template <typename TS, int B> struct DinvPad {
  static constexpr int KP = (B <= 32) ? SymPad<TS, B>::KP : Pad<TS, B>::KP;
};

// acc += M x for one packed symmetric sliced block (x a register array)
template <typename TS, typename A, int B, bool ST = true>
__device__ __forceinline__ void sym_block_mv(const TS* base, int lane, const A* x, A* acc) {
  constexpr int VW = ChunkLoad<TS, A>::VW;
  A v[VW];
#pragma unroll
  for (int j = 0; j < B; ++j) {
#pragma unroll
    for (int i = 0; i <= j; ++i) {
      const int k = j * (j + 1) / 2 + i;
      if (k % VW == 0) ChunkLoad<TS, A>::template load<ST>(base, k / VW, lane, v);
      const A m = v[k % VW];
      acc[i] += m * x[j];
      if (i != j) acc[j] += m * x[i];
    }
  }
}

// Unit kernels: one warp per slice of 32 units; the grid covers every slice.
template <int NTB>
__device__ __forceinline__ int64_t first_slice() {
  return (int64_t)blockIdx.x * (NTB / 32) + (threadIdx.x >> 5);
}

template <typename T>
struct SellView {
  const int32_t* slice_ptr;   // [nslices + 1] slot offsets
  const int32_t* cols;        // [(slot) * 32 + lane]
  const T* vals;              // [slot][KP * 32]
  int64_t nslices;
};

// Slots whose neighbour blocks are fetched together before their matrix
// blocks stream in: for small float32 blocks the column-id -> x-gather chain
// would otherwise serialise two memory latencies per slot.
#ifndef AGG_SLOT_PREFETCH
#define AGG_SLOT_PREFETCH 1
#endif
template <typename T, int B> struct SlotPrefetch {
  static constexpr int value =
      (sizeof(T) == 4 && B <= 9) ? AGG_SLOT_PREFETCH : ((sizeof(T) == 4 && B <= 16) ? 4 : 1);
};

// y_u = sum_slots A_{u,col} x_col for the thread's unit (acc zeroed by caller)
template <typename T, int B>
__device__ __forceinline__ void sell_row(const SellView<T>& A, int64_t slice, int lane, const T* __restrict__ x,
                                         T* acc) {
  constexpr int KP = Pad<T, B>::KP;
  constexpr int PF = SlotPrefetch<T, B>::value;
  const int s0 = A.slice_ptr[slice], s1 = A.slice_ptr[slice + 1];
  if constexpr (B > 32) {
    for (int j = s0; j < s1; ++j) {
      const int col = A.cols[(size_t)j * SL + lane];
      block_mv<T, T, B, 1, false>(A.vals + (size_t)j * SL * KP, lane, x + (size_t)col * B, acc);
    }
    return;
  }
  for (int j0 = s0; j0 < s1; j0 += PF) {
    const int ns = min(PF, s1 - j0);     // uniform across the warp (one slice per warp)
    int col[PF];
#pragma unroll
    for (int t = 0; t < PF; ++t) col[t] = (t < ns) ? A.cols[(size_t)(j0 + t) * SL + lane] : 0;
    T xv[PF][B];
#pragma unroll
    for (int t = 0; t < PF; ++t) {
      const T* xb = x + (size_t)col[t] * B;
#pragma unroll
      for (int c = 0; c < B; ++c) xv[t][c] = (t < ns) ? xb[c] : T(0);
    }
#pragma unroll
    for (int t = 0; t < PF; ++t)
      if (t < ns) block_mv<T, T, B, 1, false>(A.vals + (size_t)(j0 + t) * SL * KP, lane, xv[t], acc);
  }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; result valid in thread 0.
template <int NTH>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[NTH / 32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (l < NTH / 32) ? sh[l] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// Writes this block's partial; returns true in every thread of the last block
// to finish, which then owns the partials of all blocks (fixed order).
template <int NTH>
__device__ __forceinline__ bool partial_and_last(double v, double* partials, unsigned* ticket) {
  __shared__ bool last;
  double s = block_sum<NTH>(v);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

template <int NTH>
__device__ __forceinline__ double sum_partials(const double* partials, int n) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += NTH) s += ((volatile const double*)partials)[i];
  return block_sum<NTH>(s);
}

// ---------------------------------------------------------------- SpMV
// MODE 0: y = A x;  MODE 1: y = rhs - A x;  MODE 2: y = A x and (x, y) -> alpha
template <typename T, int B, int MODE, typename Op>
static __global__ void __launch_bounds__(UnitThreads<B>::value, OpMinBlocks<Op>::value)
    k_spmv(Op A, const T* __restrict__ x, const T* __restrict__ rhs, T* __restrict__ y, double* partials,
           CGState* st) {
  constexpr int NTB = UnitThreads<B>::value;
  if (st && st->done) return;
  const int lane = threadIdx.x & 31;
  double part = 0.0;
  const int64_t slice = first_slice<NTB>();
  if (slice < A.nslices()) {
    const int64_t unit = slice * SL + lane;
    T acc[B];
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] = T(0);
    A.apply(slice, lane, x, acc);
    T* yb = y + (size_t)unit * B;
#pragma unroll
    for (int r = 0; r < B; ++r) {
      if (MODE == 1) {
        yb[r] = rhs[(size_t)unit * B + r] - acc[r];
      } else {
        yb[r] = acc[r];
        if (MODE == 2) part += (double)x[(size_t)unit * B + r] * (double)acc[r];
      }
    }
  }
  if (MODE == 2) {
    if (partial_and_last<NTB>(part, partials, &st->ticket[0])) {
      double pq = sum_partials<NTB>(partials, gridDim.x);
      if (threadIdx.x == 0) {
        st->pq = pq;
        st->alpha = st->rho / pq;
        st->ticket[0] = 0;
      }
    }
  }
}

// ---------------------------------------------------------------- Chebyshev step
// KIND 0: d = c2 Dinv rhs, x_new = d                          (start from x = 0)
// KIND 1: d = c2 Dinv (rhs - A x_old), x_new = x_old + d      (first step, x given)
// KIND 2: d = c1 d + c2 Dinv (rhs - A x_old), x_new = x_old + d
// Blocks of more than 32 DoFs keep the residual in the thread's own strided
// shared-memory slot (read by that thread only) instead of registers.
template <typename T, typename TD, int B, int KIND, typename Op>
static __global__ void __launch_bounds__(UnitThreads<B>::value, OpMinBlocks<Op>::value)
    k_cheb(Op A, const TD* __restrict__ Dinv, const T* __restrict__ rhs, const T* __restrict__ x_old,
           T* __restrict__ x_new, T* __restrict__ d, T c1, T c2, int64_t nslices, const CGState* st) {
  constexpr int NTB = UnitThreads<B>::value;
  if (st && st->done) return;
  constexpr int KPD = DinvPad<TD, B>::KP;
  const int lane = threadIdx.x & 31;
  {
  const int64_t slice = first_slice<NTB>();
  if (slice >= nslices) return;
  const int64_t unit = slice * SL + lane;
  const size_t o = (size_t)unit * B;
  const TD* Db = Dinv + (size_t)slice * SL * KPD;
  T s[B];
#pragma unroll
  for (int r = 0; r < B; ++r) s[r] = T(0);
  if constexpr (B > 32) {
    __shared__ T tsh[B * NTB];
    T* ts = tsh + threadIdx.x;
    if (KIND == 0) {
      block_mv<TD, T, B, 1, OpStreams<Op>::value>(Db, lane, rhs + o, s);
    } else {
      {
        T acc[B];
#pragma unroll
        for (int r = 0; r < B; ++r) acc[r] = T(0);
        A.apply(slice, lane, x_old, acc);
#pragma unroll
        for (int r = 0; r < B; ++r) ts[r * NTB] = rhs[o + r] - acc[r];
      }
      block_mv<TD, T, B, NTB, OpStreams<Op>::value>(Db, lane, ts, s);
    }
  } else {
    T t[B];
    if (KIND == 0) {
#pragma unroll
      for (int r = 0; r < B; ++r) t[r] = rhs[o + r];
    } else {
      T acc[B];
#pragma unroll
      for (int r = 0; r < B; ++r) acc[r] = T(0);
      A.apply(slice, lane, x_old, acc);
#pragma unroll
      for (int r = 0; r < B; ++r) t[r] = rhs[o + r] - acc[r];
    }
    sym_block_mv<TD, T, B, OpStreams<Op>::value>(Db, lane, t, s);
  }
#pragma unroll
  for (int r = 0; r < B; ++r) {
    T dn = (KIND == 2) ? c1 * d[o + r] + c2 * s[r] : c2 * s[r];
    d[o + r] = dn;
    x_new[o + r] = (KIND == 0) ? dn : x_old[o + r] + dn;
  }
  }
}

// ---------------------------------------------------------------- transfers
// S_u = P_u^T (rhs_u - (A x)_u): residual of the pre-smoothed iterate, restricted
template <typename T, int B, typename Op>
static __global__ void __launch_bounds__(UnitThreads<B>::value, OpMinBlocks<Op>::value)
    k_resid_restrict(Op A, const T* __restrict__ P, const T* __restrict__ rhs, const T* __restrict__ x,
                     T* __restrict__ S, const CGState* st) {
  constexpr int NTB = UnitThreads<B>::value;
  if (st && st->done) return;
  constexpr int KP = Pad<T, B>::KP;
  const int lane = threadIdx.x & 31;
  {
  const int64_t slice = first_slice<NTB>();
  if (slice >= A.nslices()) return;
  const int64_t unit = slice * SL + lane;
  const size_t o = (size_t)unit * B;
  const T* Pb = P + (size_t)slice * SL * KP;
  T s[B];
#pragma unroll
  for (int r = 0; r < B; ++r) s[r] = T(0);
  if constexpr (B > 32) {
    T acc[B];
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] = T(0);
    A.apply(slice, lane, x, acc);
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] = rhs[o + r] - acc[r];
    block_mtv_out<T, T, B, OpStreams<Op>::value>(Pb, lane, acc, S + o);
    return;
  } else {
    T acc[B];
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] = T(0);
    A.apply(slice, lane, x, acc);
    T t[B];
#pragma unroll
    for (int r = 0; r < B; ++r) t[r] = rhs[o + r] - acc[r];
    block_mtv<T, T, B, 1, OpStreams<Op>::value>(Pb, lane, t, s);
  }
#pragma unroll
  for (int j = 0; j < B; ++j) S[o + j] = s[j];
  }
}

// rc[K*B + j] = sum over the children u of K of S[u*B + j] (children contiguous)
template <typename T, int B>
static __global__ void k_segsum(const int64_t* __restrict__ child_ptr, const T* __restrict__ S, T* __restrict__ rc,
                         int64_t nK, const CGState* st) {
  if (st && st->done) return;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nK * B) return;
  const int64_t K = id / B;
  const int j = (int)(id % B);
  T s = T(0);
#pragma unroll 4
  for (int64_t u = child_ptr[K]; u < child_ptr[K + 1]; ++u) s += S[(size_t)u * B + j];
  rc[id] = s;
}

// x_u += P_u e_{parent(u)}; ST: stream the P blocks (level 0)
template <typename T, int B, bool ST = true>
static __global__ void __launch_bounds__(UnitThreads<B>::value)
    k_prolong(const T* __restrict__ P, const int32_t* __restrict__ parent, const T* __restrict__ ec,
              T* __restrict__ x, int64_t nslices, const CGState* st) {
  constexpr int NTB = UnitThreads<B>::value;
  if (st && st->done) return;
  constexpr int KP = Pad<T, B>::KP;
  const int lane = threadIdx.x & 31;
  {
  const int64_t slice = first_slice<NTB>();
  if (slice >= nslices) return;
  const int64_t unit = slice * SL + lane;
  const size_t o = (size_t)unit * B;
  const T* eb = ec + (size_t)parent[unit] * B;
  T acc[B];
#pragma unroll
  for (int j = 0; j < B; ++j) acc[j] = T(0);
  if constexpr (B > 32) {
    block_mv<T, T, B, 1, ST>(P + (size_t)slice * SL * KP, lane, eb, acc);
  } else {
    T ev[B];
#pragma unroll
    for (int j = 0; j < B; ++j) ev[j] = eb[j];
    block_mv<T, T, B, 1, ST>(P + (size_t)slice * SL * KP, lane, ev, acc);
  }
#pragma unroll
  for (int r = 0; r < B; ++r) x[o + r] += acc[r];
  }
}

// ---------------------------------------------------------------- coarsest solve
// y = Linv r (lower triangular, row-major), one warp per row
template <typename T>
static __global__ void k_coarse_lower(const double* __restrict__ Linv, const T* __restrict__ r, double* __restrict__ y,
                               int64_t n, const CGState* st) {
  if (st && st->done) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* Lr = Linv + (size_t)row * n;
  double s = 0.0;
  // unrolled so that several loads are in flight; the sum keeps its order
#pragma unroll 8
  for (int64_t k = lane; k <= row; k += 32) s += Lr[k] * (double)r[k];
  s = warp_sum(s);
  if (lane == 0) y[row] = s;
}
// z = Linv^T y using U = Linv^T stored row-major (upper triangular)
template <typename T>
static __global__ void k_coarse_upper(const double* __restrict__ U, const double* __restrict__ y, T* __restrict__ z,
                               int64_t n, const CGState* st) {
  if (st && st->done) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* Ur = U + (size_t)row * n;
  double s = 0.0;
#pragma unroll 8
  for (int64_t k = row + lane; k < n; k += 32) s += Ur[k] * y[k];
  s = warp_sum(s);
  if (lane == 0) z[row] = (T)s;
}

}  // namespace aggmg
