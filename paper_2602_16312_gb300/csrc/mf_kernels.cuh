// Matrix-free fine-level operator (2D quadrilaterals, float32): the SIPG
// form plus mass term y = (c M + A) x evaluated element by element from
// per-quadrature-point geometry (Section 5.2: operator evaluation by
// quadrature with sum factorisation for tensor-product bases), instead of
// streaming the assembled blocks. One thread per element; it reads its own
// and its face neighbours' DoFs, the cell data G = w|J| J^-1 D J^-T and
// c w|J| at the (p+2)^2 Gauss points, and per face the reference-gradient
// flux coefficients of both sides and the weighted penalty.
//
// Face terms for the test function phi_i of element e (n: e's outward
// normal, + = e, - = neighbour; wdS folded into a, b, s):
//   -1/2 phi_i (a.grad u+ + b.grad u-) - 1/2 (a.grad phi_i) (u+ - u-) + s (u+ - u-) phi_i
#pragma once
#include "kernels.cuh"

namespace aggmg {

template <int B> struct MfDegree;
template <> struct MfDegree<4> { static constexpr int value = 1; };
template <> struct MfDegree<9> { static constexpr int value = 2; };
template <> struct MfDegree<16> { static constexpr int value = 3; };

// 1D tables: L[a][k] = l_a(x_k), D[a][k] = l_a'(x_k) at the Gauss points,
// Dend[s][a] = l_a'(s) at the end points s = 0, 1 (l_a(s) is a Kronecker
// delta on GLL nodes).
struct MfTables {
  float L[6][8];
  float D[6][8];
  float Dend[2][6];
};

struct MfView {
  const float* cell;     // [slice][qp*4 + comp][lane]
  const float* face;     // [slice][f][q*5 + comp][lane]
  const int32_t* nbr;    // [slice][f][lane]
  const int8_t* code;    // [slice][f][lane]  neighbour face * 2 + reversed
  int64_t nslices;
};

// Neighbour trace values and reference gradients at the Q face points of its
// local face (KN, SN), in its own tangential order.
template <int P, int KN, int SN>
__device__ __forceinline__ void mf_nbr_face(const MfTables& T, const float* xn, float* un, float* g0, float* g1) {
  constexpr int N = P + 1, Q = P + 2;
  const int fixed = SN * P;
  float dn[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) s += T.Dend[SN][i] * (KN == 0 ? xn[i + N * j] : xn[j + N * i]);
    dn[j] = s;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float u = 0.f, gt = 0.f, gn = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float xf = (KN == 0) ? xn[fixed + N * j] : xn[j + N * fixed];
      u += T.L[j][q] * xf;
      gt += T.D[j][q] * xf;
      gn += T.L[j][q] * dn[j];
    }
    un[q] = u;
    if (KN == 0) { g0[q] = gn; g1[q] = gt; }
    else { g0[q] = gt; g1[q] = gn; }
  }
}

template <int B>
struct MfOp {
  MfView V;
  MfTables T;
  __device__ __forceinline__ int64_t nslices() const { return V.nslices; }

  // acc += ((c M + A) x)_e for the thread's element
  __device__ __forceinline__ void apply(int64_t slice, int lane, const float* __restrict__ x, float* acc) const {
    constexpr int P = MfDegree<B>::value, N = P + 1, Q = P + 2;
    const int64_t unit = slice * SL + lane;
    float u[N * N];
#pragma unroll
    for (int i = 0; i < N * N; ++i) u[i] = x[(size_t)unit * B + i];
#ifndef AGG_MF_CELL_DIRECT
#define AGG_MF_CELL_DIRECT 0
#endif
    const float* cd = V.cell + (size_t)slice * Q * Q * 4 * SL + lane;
    if constexpr (AGG_MF_CELL_DIRECT) {
      // ---- cell term point by point: more FP32 work, few live registers
#pragma unroll 1
      for (int l = 0; l < Q; ++l) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          float uq = 0.f, g0 = 0.f, g1 = 0.f;
#pragma unroll
          for (int b = 0; b < N; ++b) {
            float su = 0.f, sd = 0.f;
#pragma unroll
            for (int a = 0; a < N; ++a) {
              su += T.L[a][k] * u[a + N * b];
              sd += T.D[a][k] * u[a + N * b];
            }
            uq += T.L[b][l] * su;
            g0 += T.L[b][l] * sd;
            g1 += T.D[b][l] * su;
          }
          const int iq = k + Q * l;
          const float G00 = __ldg(cd + (iq * 4 + 0) * SL), G01 = __ldg(cd + (iq * 4 + 1) * SL);
          const float G11 = __ldg(cd + (iq * 4 + 2) * SL), mm = __ldg(cd + (iq * 4 + 3) * SL);
          const float w0 = G00 * g0 + G01 * g1;
          const float w1 = G01 * g0 + G11 * g1;
          const float wm = mm * uq;
#pragma unroll
          for (int b = 0; b < N; ++b) {
            const float cb0 = T.L[b][l] * w0, cb1 = T.D[b][l] * w1 + T.L[b][l] * wm;
#pragma unroll
            for (int a = 0; a < N; ++a) acc[a + N * b] += T.D[a][k] * cb0 + T.L[a][k] * cb1;
          }
        }
      }
    } else {
    // ---- cell term by sum factorisation (index i = a + N b, qp = k + Q l)
    // ---- cell term by sum factorisation (index i = a + N b, qp = k + Q l)
    float tu[N][Q], td[N][Q];
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int a = 0; a < N; ++a) {
          s0 += T.L[a][k] * u[a + N * b];
          s1 += T.D[a][k] * u[a + N * b];
        }
        tu[b][k] = s0;
        td[b][k] = s1;
      }
    float p0[N][Q], p1[N][Q];
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int k = 0; k < Q; ++k) { p0[b][k] = 0.f; p1[b][k] = 0.f; }
#pragma unroll
    for (int l = 0; l < Q; ++l)
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        float uq = 0.f, g0 = 0.f, g1 = 0.f;
#pragma unroll
        for (int b = 0; b < N; ++b) {
          uq += T.L[b][l] * tu[b][k];
          g0 += T.L[b][l] * td[b][k];
          g1 += T.D[b][l] * tu[b][k];
        }
        const int iq = k + Q * l;
        const float G00 = __ldg(cd + (iq * 4 + 0) * SL), G01 = __ldg(cd + (iq * 4 + 1) * SL);
        const float G11 = __ldg(cd + (iq * 4 + 2) * SL), mm = __ldg(cd + (iq * 4 + 3) * SL);
        const float w0 = G00 * g0 + G01 * g1;
        const float w1 = G01 * g0 + G11 * g1;
        const float wm = mm * uq;
#pragma unroll
        for (int b = 0; b < N; ++b) {
          p0[b][k] += T.L[b][l] * w0;
          p1[b][k] += T.D[b][l] * w1 + T.L[b][l] * wm;
        }
      }
    // p0 carries the d/dxi0 test term, p1 the d/dxi1 and mass terms
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < Q; ++k) s += T.D[a][k] * p0[b][k] + T.L[a][k] * p1[b][k];
        acc[a + N * b] += s;
      }
    }
    // ---- face terms
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const size_t fi = ((size_t)slice * 4 + f) * SL + lane;
      const int nb = V.nbr[fi];
      if (nb < 0) continue;
      const int code = V.code[fi];
      const int fn = code >> 1, rev = code & 1;
      const int KF = f / 2, SF = f % 2;
      const int fixed = SF * P;
      // own side: trace, tangential and normal derivatives at the face points
      float dn[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < N; ++i) s += T.Dend[SF][i] * (KF == 0 ? u[i + N * j] : u[j + N * i]);
        dn[j] = s;
      }
      float xn[N * N];
#pragma unroll
      for (int i = 0; i < N * N; ++i) xn[i] = x[(size_t)nb * B + i];
      float un[Q], gn0[Q], gn1[Q];
      switch (fn) {
        case 0: mf_nbr_face<P, 0, 0>(T, xn, un, gn0, gn1); break;
        case 1: mf_nbr_face<P, 0, 1>(T, xn, un, gn0, gn1); break;
        case 2: mf_nbr_face<P, 1, 0>(T, xn, un, gn0, gn1); break;
        default: mf_nbr_face<P, 1, 1>(T, xn, un, gn0, gn1); break;
      }
      const float* fd = V.face + (size_t)((slice * 4 + f) * Q * 5) * SL + lane;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        float up = 0.f, gt = 0.f, gn = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float xf = (KF == 0) ? u[fixed + N * j] : u[j + N * fixed];
          up += T.L[j][q] * xf;
          gt += T.D[j][q] * xf;
          gn += T.L[j][q] * dn[j];
        }
        const float g0p = (KF == 0) ? gn : gt;
        const float g1p = (KF == 0) ? gt : gn;
        const float a0 = __ldg(fd + (q * 5 + 0) * SL), a1 = __ldg(fd + (q * 5 + 1) * SL);
        const float b0 = __ldg(fd + (q * 5 + 2) * SL), b1 = __ldg(fd + (q * 5 + 3) * SL);
        const float sq = __ldg(fd + (q * 5 + 4) * SL);
        const float um = rev ? un[Q - 1 - q] : un[q];
        const float h0 = rev ? gn0[Q - 1 - q] : gn0[q];
        const float h1 = rev ? gn1[Q - 1 - q] : gn1[q];
        const float flux = a0 * g0p + a1 * g1p + b0 * h0 + b1 * h1;
        const float jump = up - um;
        const float cf = -0.5f * flux + sq * jump;     // times phi_i on the face
        const float cn = -0.5f * jump * (KF == 0 ? a0 : a1);   // times d phi_i / d xi_normal
        const float ct = -0.5f * jump * (KF == 0 ? a1 : a0);   // times d phi_i / d xi_tangential
#pragma unroll
        for (int j = 0; j < N; ++j) {
          // face DoFs: value and tangential derivative
          const int idf = (KF == 0) ? fixed + N * j : j + N * fixed;
          acc[idf] += T.L[j][q] * cf + T.D[j][q] * ct;
          // normal derivative of every DoF on the line j
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const int id = (KF == 0) ? i + N * j : j + N * i;
            acc[id] += T.Dend[SF][i] * T.L[j][q] * cn;
          }
        }
      }
    }
  }
};

// Sliced block-sparse operator in the same interface.
template <typename T, int B>
struct SellOp {
  SellView<T> A;
  __device__ __forceinline__ int64_t nslices() const { return A.nslices; }
  __device__ __forceinline__ void apply(int64_t slice, int lane, const T* __restrict__ x, T* acc) const {
    sell_row<T, B>(A, slice, lane, x, acc);
  }
};

// y = op x for a unit-kernel operator (used to test an operator on its own)
template <typename T, int B, typename Op>
static __global__ void __launch_bounds__(UnitThreads<B>::value) k_op_apply(Op op, const T* __restrict__ x,
                                                                          T* __restrict__ y) {
  constexpr int NTB = UnitThreads<B>::value;
  const int lane = threadIdx.x & 31;
  {
  const int64_t slice = first_slice<NTB>();
  if (slice >= op.nslices()) return;
    T acc[B];
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] = T(0);
    op.apply(slice, lane, x, acc);
    const size_t o = (size_t)(slice * SL + lane) * B;
#pragma unroll
    for (int r = 0; r < B; ++r) y[o + r] = acc[r];
  }
}

}  // namespace aggmg
