// Face-structured assembled operator of level 0 (float64 for the outer CG,
// the V-cycle precision for the smoother): the dense diagonal block of each
// element and, per local face f, only the parts of the coupling block that
// a GLL nodal basis can make nonzero. A basis function whose node is off a
// face vanishes on it, so the SIPG face terms between e and its neighbour n
// (Section 3, Eq. bilinear_form: consistency, symmetry and penalty terms)
// touch
//   R_f: e's rows on face f  x  all columns of n   (trace of e's test function)
//   C_f: e's other rows      x  n's columns on its face fn (trace of n's trial function)
// i.e. 2 NF B - NF^2 of the B^2 entries (NF = N^(d-1) face DoFs): 405 of 729
// for Q2 hexahedra, 1792 of 4096 for Q3. The arithmetic is the block product
// with the structural zeros skipped.
#pragma once
#include "kernels.cuh"

namespace aggmg {

template <int B> struct FaceShape;
template <> struct FaceShape<4> { static constexpr int D = 2, N = 2; };
template <> struct FaceShape<9> { static constexpr int D = 2, N = 3; };
template <> struct FaceShape<16> { static constexpr int D = 2, N = 4; };
template <> struct FaceShape<8> { static constexpr int D = 3, N = 2; };
template <> struct FaceShape<27> { static constexpr int D = 3, N = 3; };
template <> struct FaceShape<64> { static constexpr int D = 3, N = 4; };

// DoF indices (i = a + N b [+ N^2 c]) on and off local face f = 2k + s.
// Face DoF r = j1 + N j2 over the tangential axes in increasing order; off-face
// DoF r = j1 + N j2 + NF i' with i' the normal index with the face layer
// left out.
template <int D, int N>
struct FaceIdx {
  static constexpr int NN = N * N, NF = (D == 2) ? N : NN;
  __device__ __forceinline__ static int stride(int a) { return a == 0 ? 1 : (a == 1 ? N : NN); }
  __device__ __forceinline__ static int tang(int k, int r) {
    if constexpr (D == 2) return r * stride(1 - k);
    return (r % N) * stride(k == 0 ? 1 : 0) + (r / N) * stride(k == 2 ? 1 : 2);
  }
  __device__ __forceinline__ static int face(int f, int r) {
    return (f & 1) * (N - 1) * stride(f >> 1) + tang(f >> 1, r);
  }
  __device__ __forceinline__ static int off(int f, int r) {
    return (r / NF + 1 - (f & 1)) * stride(f >> 1) + tang(f >> 1, r % NF);
  }
};

// acc[om(r)] += sum_c M[r][c] x(c) for one sliced ROWS x COLS block stored
// column-major (k = c ROWS + r) in chunks of VW. Large blocks loop over the
// columns at run time (rows unrolled), so om(r) stays a constant.
template <typename TS, typename A, int ROWS, int COLS, typename XF, typename OM>
__device__ __forceinline__ void rect_mv(const TS* base, int lane, XF x, OM om, A* acc) {
  constexpr int VW = ChunkLoad<TS, A>::VW;
  if constexpr (ROWS * COLS > 512 && ROWS % VW == 0) {
#pragma unroll 1
    for (int c = 0; c < COLS; ++c) {
      const A xc = x(c);
#pragma unroll
      for (int rr = 0; rr < ROWS / VW; ++rr) {
        A v[VW];
        ChunkLoad<TS, A>::load(base, c * (ROWS / VW) + rr, lane, v);
#pragma unroll
        for (int t = 0; t < VW; ++t) acc[om(rr * VW + t)] += v[t] * xc;
      }
    }
  } else {
    constexpr int NCH = (ROWS * COLS + VW - 1) / VW;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      A v[VW];
      ChunkLoad<TS, A>::load(base, ch, lane, v);
#pragma unroll
      for (int t = 0; t < VW; ++t) {
        const int k = ch * VW + t;
        if (k < ROWS * COLS) acc[om(k % ROWS)] += v[t] * x(k / ROWS);
      }
    }
  }
}

template <typename T, int B>
struct FaceView {
  const T* vals;          // per slice: diagonal block, then per face R_f and C_f
  const int32_t* nbr;     // [slice][f][lane] neighbour's internal index or -1
  const int8_t* code;     // [slice][f][lane] neighbour's local face
  int64_t nslices;
};

template <typename T, int B>
struct FaceOp {
  static constexpr int D = FaceShape<B>::D, N = FaceShape<B>::N;
  using FI = FaceIdx<D, N>;
  static constexpr int NF = FI::NF, NFACE = 2 * D, BO = B - NF;
  static constexpr int VW = Vec<T>::W;
  static constexpr int KP = Pad<T, B>::KP;
  static constexpr int KR = ((NF * B + VW - 1) / VW) * VW;
  static constexpr int KC = ((BO * NF + VW - 1) / VW) * VW;
  static constexpr int KS = KP + NFACE * (KR + KC);   // values per lane and slice
  FaceView<T, B> V;
  __device__ __forceinline__ int64_t nslices() const { return V.nslices; }

  // acc += (A x)_u for the thread's unit
  __device__ __forceinline__ void apply(int64_t slice, int lane, const T* __restrict__ x, T* acc) const {
    const T* base = V.vals + (size_t)slice * SL * KS;
    const T* xe = x + (size_t)(slice * SL + lane) * B;
    if constexpr (B > 32) {
      block_mv<T, T, B>(base, lane, xe, acc);
    } else {
      T xr[B];
#pragma unroll
      for (int c = 0; c < B; ++c) xr[c] = xe[c];
      block_mv<T, T, B>(base, lane, xr, acc);
    }
#pragma unroll
    for (int f = 0; f < NFACE; ++f) {
      const size_t fi = ((size_t)slice * NFACE + f) * SL + lane;
      const int nb = V.nbr[fi];
      if (nb < 0) continue;
      const int fn = V.code[fi];
      const T* xn = x + (size_t)nb * B;
      const T* Rb = base + (size_t)SL * (KP + f * (KR + KC));
      const T* Cb = Rb + (size_t)SL * KR;
      auto on_face = [&](int r) { return FI::face(f, r); };
      auto off_face = [&](int r) { return FI::off(f, r); };
      if constexpr (B > 32) {
        rect_mv<T, T, NF, B>(Rb, lane, [&](int c) { return xn[c]; }, on_face, acc);
        rect_mv<T, T, BO, NF>(Cb, lane, [&](int c) { return xn[FI::face(fn, c)]; }, off_face, acc);
      } else {
        T xv[B], xf[NF];
#pragma unroll
        for (int c = 0; c < B; ++c) xv[c] = xn[c];
#pragma unroll
        for (int j = 0; j < NF; ++j) xf[j] = xn[FI::face(fn, j)];
        rect_mv<T, T, NF, B>(Rb, lane, [&](int c) { return xv[c]; }, on_face, acc);
        rect_mv<T, T, BO, NF>(Cb, lane, [&](int c) { return xf[c]; }, off_face, acc);
      }
    }
  }
};

}  // namespace aggmg
