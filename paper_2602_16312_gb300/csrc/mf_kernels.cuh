// Matrix-free fine-level operator (quadrilaterals, hexahedra; float32): the SIPG
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
template <typename R>
struct MfTablesT {
  R L[6][8];
  R D[6][8];
  R Dend[2][6];
};
using MfTables = MfTablesT<float>;

template <typename R>
struct MfViewT {
  const R* cell;         // [slice][qp*4 + comp][lane]
  const R* face;         // [slice][f][q*5 + comp][lane]
  const int32_t* nbr;    // [slice][f][lane]
  const int8_t* code;    // [slice][f][lane]  neighbour face * 2 + reversed
  int64_t nslices;
};
using MfView = MfViewT<float>;

// Neighbour trace values and reference gradients at the Q face points of its
// local face (KN, SN), in its own tangential order.
template <typename R, int P, int KN, int SN>
__device__ __forceinline__ void mf_nbr_face(const MfTablesT<R>& T, const R* xn, R* un, R* g0, R* g1) {
  constexpr int N = P + 1, Q = P + 2;
  const int fixed = SN * P;
  R dn[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < N; ++i) s += T.Dend[SN][i] * (KN == 0 ? xn[i + N * j] : xn[j + N * i]);
    dn[j] = s;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    R u = R(0), gt = R(0), gn = R(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const R xf = (KN == 0) ? xn[fixed + N * j] : xn[j + N * fixed];
      u += T.L[j][q] * xf;
      gt += T.D[j][q] * xf;
      gn += T.L[j][q] * dn[j];
    }
    un[q] = u;
    if (KN == 0) { g0[q] = gn; g1[q] = gt; }
    else { g0[q] = gt; g1[q] = gn; }
  }
}

// Minimum resident blocks of 128 threads asked of the compiler for the 2D
// operator's kernels (AGG_MF2_MINB overrides it; 0 leaves the registers
// free). Float32 Q2: 7 blocks (72 registers, 12 B spilled) ran the
// Chebyshev step in 57.0 instead of 58.2 us (80 registers, 6 blocks) on the
// 512^2 square, three runs each on one GB300; 8 blocks spilled 156 B and
// took 85 us.
#ifndef AGG_MF2_MINB
#define AGG_MF2_MINB -1
#endif
template <typename R, int B> struct Mf2MinBlocks { static constexpr int value = 0; };
template <> struct Mf2MinBlocks<float, 9> { static constexpr int value = 7; };
#ifndef AGG_MF2_DIRECT_BACK
#define AGG_MF2_DIRECT_BACK 0
#endif
template <typename R, int B>
struct MfOpV {
  static constexpr int kDegree = MfDegree<B>::value;
  static constexpr int kMinBlocks = (AGG_MF2_MINB >= 0) ? AGG_MF2_MINB : Mf2MinBlocks<R, B>::value;
  MfViewT<R> V;
  MfTablesT<R> T;
  __device__ __forceinline__ int64_t nslices() const { return V.nslices; }

  // acc += ((c M + A) x)_e for the thread's element
  __device__ __forceinline__ void apply(int64_t slice, int lane, const R* __restrict__ x, R* acc) const {
    constexpr int N = MfDegree<B>::value + 1;
    const int64_t unit = slice * SL + lane;
    R u[N * N];
#pragma unroll
    for (int i = 0; i < N * N; ++i) u[i] = x[(size_t)unit * B + i];
    cell(slice, lane, u, acc);
    faces(slice, lane, x, u, acc);
  }

  // acc += the cell (volume and mass) terms of the element whose DoFs are u;
  // DB: back-project each Gauss point straight into acc (more FMAs, no
  // partial sums held in registers)
  template <bool DB = (AGG_MF2_DIRECT_BACK != 0)>
  __device__ __forceinline__ void cell(int64_t slice, int lane, const R* u, R* acc) const {
    constexpr int P = MfDegree<B>::value, N = P + 1, Q = P + 2;
#ifndef AGG_MF_CELL_DIRECT
#define AGG_MF_CELL_DIRECT 0
#endif
    const R* cd = V.cell + (size_t)slice * Q * Q * 4 * SL + lane;
    if constexpr (AGG_MF_CELL_DIRECT) {
      // ---- cell term point by point: more FP32 work, few live registers
#pragma unroll 1
      for (int l = 0; l < Q; ++l) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          R uq = R(0), g0 = R(0), g1 = R(0);
#pragma unroll
          for (int b = 0; b < N; ++b) {
            R su = R(0), sd = R(0);
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
          const R G00 = ld_once(cd + (iq * 4 + 0) * SL), G01 = ld_once(cd + (iq * 4 + 1) * SL);
          const R G11 = ld_once(cd + (iq * 4 + 2) * SL), mm = ld_once(cd + (iq * 4 + 3) * SL);
          const R w0 = G00 * g0 + G01 * g1;
          const R w1 = G01 * g0 + G11 * g1;
          const R wm = mm * uq;
#pragma unroll
          for (int b = 0; b < N; ++b) {
            const R cb0 = T.L[b][l] * w0, cb1 = T.D[b][l] * w1 + T.L[b][l] * wm;
#pragma unroll
            for (int a = 0; a < N; ++a) acc[a + N * b] += T.D[a][k] * cb0 + T.L[a][k] * cb1;
          }
        }
      }
    } else {
    // ---- cell term by sum factorisation (index i = a + N b, qp = k + Q l)
    R tu[N][Q], td[N][Q];
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        R s0 = R(0), s1 = R(0);
#pragma unroll
        for (int a = 0; a < N; ++a) {
          s0 += T.L[a][k] * u[a + N * b];
          s1 += T.D[a][k] * u[a + N * b];
        }
        tu[b][k] = s0;
        td[b][k] = s1;
      }
    if constexpr (DB) {
      // back-projection of each Gauss point straight into acc (more FMAs,
      // no p0/p1 partial sums held in registers)
#pragma unroll
      for (int l = 0; l < Q; ++l)
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          R uq = R(0), g0 = R(0), g1 = R(0);
#pragma unroll
          for (int b = 0; b < N; ++b) {
            uq += T.L[b][l] * tu[b][k];
            g0 += T.L[b][l] * td[b][k];
            g1 += T.D[b][l] * tu[b][k];
          }
          const int iq = k + Q * l;
          const R G00 = ld_once(cd + (iq * 4 + 0) * SL), G01 = ld_once(cd + (iq * 4 + 1) * SL);
          const R G11 = ld_once(cd + (iq * 4 + 2) * SL), mm = ld_once(cd + (iq * 4 + 3) * SL);
          const R w0 = G00 * g0 + G01 * g1;
          const R w1 = G01 * g0 + G11 * g1;
          const R wm = mm * uq;
#pragma unroll
          for (int b = 0; b < N; ++b) {
            const R cb0 = T.L[b][l] * w0, cb1 = T.D[b][l] * w1 + T.L[b][l] * wm;
#pragma unroll
            for (int a = 0; a < N; ++a) acc[a + N * b] += T.D[a][k] * cb0 + T.L[a][k] * cb1;
          }
        }
    } else {
    R p0[N][Q], p1[N][Q];
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int k = 0; k < Q; ++k) { p0[b][k] = R(0); p1[b][k] = R(0); }
#pragma unroll
    for (int l = 0; l < Q; ++l)
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        R uq = R(0), g0 = R(0), g1 = R(0);
#pragma unroll
        for (int b = 0; b < N; ++b) {
          uq += T.L[b][l] * tu[b][k];
          g0 += T.L[b][l] * td[b][k];
          g1 += T.D[b][l] * tu[b][k];
        }
        const int iq = k + Q * l;
        const R G00 = ld_once(cd + (iq * 4 + 0) * SL), G01 = ld_once(cd + (iq * 4 + 1) * SL);
        const R G11 = ld_once(cd + (iq * 4 + 2) * SL), mm = ld_once(cd + (iq * 4 + 3) * SL);
        const R w0 = G00 * g0 + G01 * g1;
        const R w1 = G01 * g0 + G11 * g1;
        const R wm = mm * uq;
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
        R s = R(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) s += T.D[a][k] * p0[b][k] + T.L[a][k] * p1[b][k];
        acc[a + N * b] += s;
      }
    }
    }
  }

  // acc += the face terms of the element whose DoFs are u (x: all DoFs, for
  // the neighbours)
  __device__ __forceinline__ void faces(int64_t slice, int lane, const R* __restrict__ x, const R* u, R* acc) const {
    constexpr int P = MfDegree<B>::value, N = P + 1, Q = P + 2;
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
      R dn[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        R s = R(0);
#pragma unroll
        for (int i = 0; i < N; ++i) s += T.Dend[SF][i] * (KF == 0 ? u[i + N * j] : u[j + N * i]);
        dn[j] = s;
      }
      R xn[N * N];
#pragma unroll
      for (int i = 0; i < N * N; ++i) xn[i] = x[(size_t)nb * B + i];
      R un[Q], gn0[Q], gn1[Q];
      switch (fn) {
        case 0: mf_nbr_face<R, P, 0, 0>(T, xn, un, gn0, gn1); break;
        case 1: mf_nbr_face<R, P, 0, 1>(T, xn, un, gn0, gn1); break;
        case 2: mf_nbr_face<R, P, 1, 0>(T, xn, un, gn0, gn1); break;
        default: mf_nbr_face<R, P, 1, 1>(T, xn, un, gn0, gn1); break;
      }
      const R* fd = V.face + (size_t)((slice * 4 + f) * Q * 5) * SL + lane;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        R up = R(0), gt = R(0), gn = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const R xf = (KF == 0) ? u[fixed + N * j] : u[j + N * fixed];
          up += T.L[j][q] * xf;
          gt += T.D[j][q] * xf;
          gn += T.L[j][q] * dn[j];
        }
        const R g0p = (KF == 0) ? gn : gt;
        const R g1p = (KF == 0) ? gt : gn;
        const R a0 = ld_once(fd + (q * 5 + 0) * SL), a1 = ld_once(fd + (q * 5 + 1) * SL);
        const R b0 = ld_once(fd + (q * 5 + 2) * SL), b1 = ld_once(fd + (q * 5 + 3) * SL);
        const R sq = ld_once(fd + (q * 5 + 4) * SL);
        const R um = rev ? un[Q - 1 - q] : un[q];
        const R h0 = rev ? gn0[Q - 1 - q] : gn0[q];
        const R h1 = rev ? gn1[Q - 1 - q] : gn1[q];
        const R flux = a0 * g0p + a1 * g1p + b0 * h0 + b1 * h1;
        const R jump = up - um;
        const R cf = R(-0.5) * flux + sq * jump;     // times phi_i on the face
        const R cn = R(-0.5) * jump * (KF == 0 ? a0 : a1);   // times d phi_i / d xi_normal
        const R ct = R(-0.5) * jump * (KF == 0 ? a1 : a0);   // times d phi_i / d xi_tangential
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

// 3D hexahedra (p = 1, 2), same scheme: cell term plane by plane (xi_2 Gauss
// plane m outermost) with sum factorisation inside the plane; face terms
// from the face traces of both sides. Planes and faces are loops at run time
// (fully unrolled, the code outgrows the instruction cache). Both sides'
// DoFs are read through strides set by the local face, and the flux
// coefficients of each side are stored in that side's face frame (normal
// axis, then the tangential axes in increasing order), so no register array
// is indexed at run time. Index i = a + N b + N^2 c, qp = k + Q l + Q^2 m.
template <int B> struct Mf3Degree;
template <> struct Mf3Degree<8> { static constexpr int value = 1; };
template <> struct Mf3Degree<27> { static constexpr int value = 2; };
template <> struct Mf3Degree<64> { static constexpr int value = 3; };

#ifndef AGG_MF3_MINB
#define AGG_MF3_MINB 0
#endif
template <typename R, int B>
struct MfOp3V {
  static constexpr int kDegree = Mf3Degree<B>::value;
  static constexpr int kMinBlocks = AGG_MF3_MINB;
  MfViewT<R> V;
  MfTablesT<R> T;
  __device__ __forceinline__ int64_t nslices() const { return V.nslices; }

  __device__ __forceinline__ void apply(int64_t slice, int lane, const R* __restrict__ x, R* acc) const {
    constexpr int P = kDegree, N = P + 1, Q = P + 2, NN = N * N, QQ = Q * Q;
    const int64_t unit = slice * SL + lane;
    R u[B];
#pragma unroll
    for (int i = 0; i < B; ++i) u[i] = x[(size_t)unit * B + i];
    const R* cd = V.cell + (size_t)slice * QQ * Q * 7 * SL + lane;
    // The test-side sums of the face terms (and for B = 64 those of the cell
    // term too) go to the thread's column of a shared array: no register
    // array is indexed at run time, and for B = 64 the 64 sums are not held
    // in registers through the plane loop (254 instead of 255 registers with
    // 136 B spilled; the 48^3 Q3 step 918 instead of 1,035 us). For B = 27
    // the same change cut the Chebyshev step by 0.7% but slowed the time step
    // of the 64^3 cube by 1%, so the cell sums stay in registers there.
    // They join acc at the end.
    constexpr bool kCellShared = (B == 64);
    constexpr int NT = UnitThreads<B>::value;
    __shared__ R sacc[B][NT];
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < B; ++i) sacc[i][t] = R(0);
    // ---- cell term
#ifndef AGG_MF3_PLANE_UNROLL
#define AGG_MF3_PLANE_UNROLL 1
#endif
    constexpr int kPlaneUnroll = AGG_MF3_PLANE_UNROLL;
#pragma unroll kPlaneUnroll
    for (int m = 0; m < Q; ++m) {
      R Lm[N], Dm[N];
#pragma unroll
      for (int c = 0; c < N; ++c) {
        Lm[c] = T.L[c][m];
        Dm[c] = T.D[c][m];
      }
      R v[NN], w[NN];
#pragma unroll
      for (int ab = 0; ab < NN; ++ab) {
        R s0 = R(0), s1 = R(0);
#pragma unroll
        for (int c = 0; c < N; ++c) {
          s0 += Lm[c] * u[ab + NN * c];
          s1 += Dm[c] * u[ab + NN * c];
        }
        v[ab] = s0;
        w[ab] = s1;
      }
      R tu[N][Q], td[N][Q], tw[N][Q];
#pragma unroll
      for (int b = 0; b < N; ++b)
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          R s0 = R(0), s1 = R(0), s2 = R(0);
#pragma unroll
          for (int a = 0; a < N; ++a) {
            s0 += T.L[a][k] * v[a + N * b];
            s1 += T.D[a][k] * v[a + N * b];
            s2 += T.L[a][k] * w[a + N * b];
          }
          tu[b][k] = s0;
          td[b][k] = s1;
          tw[b][k] = s2;
        }
      R p0[N][Q], p1[N][Q], p2[N][Q];
#pragma unroll
      for (int b = 0; b < N; ++b)
#pragma unroll
        for (int k = 0; k < Q; ++k) { p0[b][k] = R(0); p1[b][k] = R(0); p2[b][k] = R(0); }
#pragma unroll
      for (int l = 0; l < Q; ++l)
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          R uq = R(0), g0 = R(0), g1 = R(0), g2 = R(0);
#pragma unroll
          for (int b = 0; b < N; ++b) {
            uq += T.L[b][l] * tu[b][k];
            g0 += T.L[b][l] * td[b][k];
            g1 += T.D[b][l] * tu[b][k];
            g2 += T.L[b][l] * tw[b][k];
          }
          const R* gq = cd + (size_t)((k + Q * l + QQ * m) * 7) * SL;
          const R G00 = ld_once(gq), G01 = ld_once(gq + SL), G02 = ld_once(gq + 2 * SL);
          const R G11 = ld_once(gq + 3 * SL), G12 = ld_once(gq + 4 * SL), G22 = ld_once(gq + 5 * SL);
          const R mm = ld_once(gq + 6 * SL);
          const R w0 = G00 * g0 + G01 * g1 + G02 * g2;
          const R w1 = G01 * g0 + G11 * g1 + G12 * g2;
          const R w2 = G02 * g0 + G12 * g1 + G22 * g2;
          const R wm = mm * uq;
#pragma unroll
          for (int b = 0; b < N; ++b) {
            p0[b][k] += T.L[b][l] * w0;
            p1[b][k] += T.D[b][l] * w1 + T.L[b][l] * wm;
            p2[b][k] += T.L[b][l] * w2;
          }
        }
#pragma unroll
      for (int b = 0; b < N; ++b)
#pragma unroll
        for (int a = 0; a < N; ++a) {
          R pv = R(0), pw = R(0);
#pragma unroll
          for (int k = 0; k < Q; ++k) {
            pv += T.D[a][k] * p0[b][k] + T.L[a][k] * p1[b][k];
            pw += T.L[a][k] * p2[b][k];
          }
#pragma unroll
          for (int c = 0; c < N; ++c) {
            if constexpr (kCellShared) sacc[a + N * b + NN * c][t] += Lm[c] * pv + Dm[c] * pw;
            else acc[a + N * b + NN * c] += Lm[c] * pv + Dm[c] * pw;
          }
        }
    }
    // ---- face terms: one pass per face at run time; both sides' traces are
    // read from memory through strides
    const R* xe = x + (size_t)unit * B;
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
      const size_t fi = ((size_t)slice * 6 + f) * SL + lane;
      const int nb = V.nbr[fi];
      if (nb < 0) continue;
      const int fnb = V.code[fi];
      R sU[N][Q], sT[N][Q], sN[N][Q], nU[N][Q], nT[N][Q], nN[N][Q];
      face_trace(xe, f, sU, sT, sN);
      face_trace(x + (size_t)nb * B, fnb, nU, nT, nN);
      R rF[N][Q], rT[N][Q], rN[N][Q];
#pragma unroll
      for (int j2 = 0; j2 < N; ++j2)
#pragma unroll
        for (int q1 = 0; q1 < Q; ++q1) { rF[j2][q1] = R(0); rT[j2][q1] = R(0); rN[j2][q1] = R(0); }
      const R* fd = V.face + (size_t)((slice * 6 + f) * QQ * 7) * SL + lane;
#pragma unroll
      for (int q2 = 0; q2 < Q; ++q2)
#pragma unroll
        for (int q1 = 0; q1 < Q; ++q1) {
          R up = R(0), gt0 = R(0), gt1 = R(0), gnn = R(0), um = R(0), ht0 = R(0), ht1 = R(0), hn = R(0);
#pragma unroll
          for (int j2 = 0; j2 < N; ++j2) {
            up += T.L[j2][q2] * sU[j2][q1];
            gt0 += T.L[j2][q2] * sT[j2][q1];
            gt1 += T.D[j2][q2] * sU[j2][q1];
            gnn += T.L[j2][q2] * sN[j2][q1];
            um += T.L[j2][q2] * nU[j2][q1];
            ht0 += T.L[j2][q2] * nT[j2][q1];
            ht1 += T.D[j2][q2] * nU[j2][q1];
            hn += T.L[j2][q2] * nN[j2][q1];
          }
          const R* fq = fd + (size_t)((q1 + Q * q2) * 7) * SL;
          const R aN = ld_once(fq), aT0 = ld_once(fq + SL), aT1 = ld_once(fq + 2 * SL);
          const R bN = ld_once(fq + 3 * SL), bT0 = ld_once(fq + 4 * SL), bT1 = ld_once(fq + 5 * SL);
          const R sq = ld_once(fq + 6 * SL);
          const R flux = aN * gnn + aT0 * gt0 + aT1 * gt1 + bN * hn + bT0 * ht0 + bT1 * ht1;
          const R jump = up - um;
          const R cf = R(-0.5) * flux + sq * jump;
          const R hj = R(-0.5) * jump;
#pragma unroll
          for (int j2 = 0; j2 < N; ++j2) {
            rF[j2][q1] += T.L[j2][q2] * cf + T.D[j2][q2] * (hj * aT1);
            rT[j2][q1] += T.L[j2][q2] * (hj * aT0);
            rN[j2][q1] += T.L[j2][q2] * (hj * aN);
          }
        }
      // test side: face DoFs (value, tangential derivatives) and the normal
      // derivative of every DoF behind each face node
      const int KF = f >> 1, SF = f & 1;
      const int SK = (KF == 0) ? 1 : (KF == 1 ? N : NN);
      const int S0 = (KF == 0) ? N : 1, S1 = (KF == 2) ? N : NN;
#pragma unroll
      for (int j2 = 0; j2 < N; ++j2)
#pragma unroll
        for (int j1 = 0; j1 < N; ++j1) {
          R ff = R(0), fnrm = R(0);
#pragma unroll
          for (int q1 = 0; q1 < Q; ++q1) {
            ff += T.L[j1][q1] * rF[j2][q1] + T.D[j1][q1] * rT[j2][q1];
            fnrm += T.L[j1][q1] * rN[j2][q1];
          }
          const int line = j1 * S0 + j2 * S1;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const R de = SF ? T.Dend[1][i] : T.Dend[0][i];
            const bool on_face = (SF ? P : 0) == i;
            sacc[i * SK + line][t] += de * fnrm + (on_face ? ff : R(0));
          }
        }
    }
#pragma unroll
    for (int i = 0; i < B; ++i) acc[i] += sacc[i][t];
  }

  // Trace (U), derivative along the first tangential axis (Tn) and normal
  // derivative (Nr) on local face f of the element whose DoFs start at xb,
  // interpolated to the Gauss points along the first tangential axis and
  // kept at the nodes along the second: [j2][q1].
  __device__ __forceinline__ void face_trace(const R* __restrict__ xb, int f, R (&U)[kDegree + 1][kDegree + 2],
                                             R (&Tn)[kDegree + 1][kDegree + 2],
                                             R (&Nr)[kDegree + 1][kDegree + 2]) const {
    constexpr int P = kDegree, N = P + 1, Q = P + 2, NN = N * N;
    const int k = f >> 1, sd = f & 1;
    const int SK = (k == 0) ? 1 : (k == 1 ? N : NN);
    const int S0 = (k == 0) ? N : 1, S1 = (k == 2) ? N : NN;
    const R* xf = xb + sd * P * SK;
#pragma unroll
    for (int j2 = 0; j2 < N; ++j2) {
      R tr[N], dn[N];
#pragma unroll
      for (int j1 = 0; j1 < N; ++j1) {
        R s = R(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const R de = sd ? T.Dend[1][i] : T.Dend[0][i];
          s += de * xb[i * SK + j1 * S0 + j2 * S1];
        }
        dn[j1] = s;
        tr[j1] = xf[j1 * S0 + j2 * S1];
      }
#pragma unroll
      for (int q1 = 0; q1 < Q; ++q1) {
        R a0 = R(0), a1 = R(0), a2 = R(0);
#pragma unroll
        for (int j1 = 0; j1 < N; ++j1) {
          a0 += T.L[j1][q1] * tr[j1];
          a1 += T.D[j1][q1] * tr[j1];
          a2 += T.L[j1][q1] * dn[j1];
        }
        U[j2][q1] = a0;
        Tn[j2][q1] = a1;
        Nr[j2][q1] = a2;
      }
    }
  }
};

template <int B> using MfOp = MfOpV<float, B>;
template <int B> using MfOp3 = MfOp3V<float, B>;
// matrix-free operator of value type R for B DoFs per element
template <typename R, int B> struct MfOpForT { using type = MfOpV<R, B>; };
template <typename R> struct MfOpForT<R, 8> { using type = MfOp3V<R, 8>; };
template <typename R> struct MfOpForT<R, 27> { using type = MfOp3V<R, 27>; };
template <typename R> struct MfOpForT<R, 64> { using type = MfOp3V<R, 64>; };
template <int B> struct MfOpFor { using type = typename MfOpForT<float, B>::type; };

// Sliced block-sparse operator in the same interface.
template <typename T, int B>
struct SellOp {
  SellView<T> A;
  __device__ __forceinline__ int64_t nslices() const { return A.nslices; }
  __device__ __forceinline__ void apply(int64_t slice, int lane, const T* __restrict__ x, T* acc) const {
    sell_row<T, B>(A, slice, lane, x, acc);
  }
};
template <typename T, int B> struct OpStreams<SellOp<T, B>> {
  static constexpr bool value = false;
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
