// Host float64 assembly of the SIPG-DG operator (Section 3 of arXiv 2602.16312):
// reference element tables, element mass/stiffness blocks, face matching and
// the interior-face terms of a_h, assembled as a block-CSR matrix in element
// order. Parallel over elements with OpenMP; every block row is written by
// the thread that owns the element, so the result does not depend on the
// thread count.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include "setup.h"
#include "../../include/aggmg.h"

namespace aggmg {

// ---------------------------------------------------------------- 1D tables
// Legendre P_n(x) and P_n'(x) on [-1, 1] by the three-term recurrence.
static void legendre(int n, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = n * (x * p1 - p0) / (x * x - 1.0);
}

Tables1D make_tables(int p, int q) {
  Tables1D t;
  t.p = p;
  t.q = q;
  // Gauss-Legendre: Newton on P_q from the standard asymptotic starting values
  std::vector<double> x(q), w(q);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(q, z, P, dP);
      double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    double P, dP;
    legendre(q, z, P, dP);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
  std::vector<int> ord(q);
  for (int i = 0; i < q; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return x[a] < x[b]; });
  for (int i = 0; i < q; ++i) {
    t.gx.push_back(0.5 * (x[ord[i]] + 1.0));
    t.gw.push_back(0.5 * w[ord[i]]);
  }
  // Gauss-Lobatto: end points and the roots of P_p', Newton with
  // P_p'' = (2 x P_p' - p(p+1) P_p) / (1 - x^2) (Legendre's equation)
  std::vector<double> g;
  g.push_back(-1.0);
  for (int i = p - 1; i >= 1; --i) {
    double z = std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, z, P, dP);
      double d2P = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
      double dz = dP / d2P;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    g.push_back(z);
  }
  g.push_back(1.0);
  std::sort(g.begin(), g.end());
  for (double z : g) t.gll.push_back(0.5 * (z + 1.0));
  return t;
}

void lagrange_eval(const double* nodes, int n, double x, double* v, double* d) {
  for (int i = 0; i < n; ++i) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != i) prod *= (x - nodes[m]) / (nodes[i] - nodes[m]);
    v[i] = prod;
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == i) continue;
      double term = 1.0 / (nodes[i] - nodes[k]);
      for (int m = 0; m < n; ++m)
        if (m != i && m != k) term *= (x - nodes[m]) / (nodes[i] - nodes[m]);
      s += term;
    }
    d[i] = s;
  }
}

// ---------------------------------------------------------------- element geometry
namespace {

constexpr int MAXD = 3;
constexpr int MAXB = 125;   // (4+1)^3

struct Basis {               // tensor basis values and reference gradients at one point
  double phi[MAXB];
  double g[MAXB][MAXD];
};

void tensor_basis(const Tables1D& t, int dim, const double* xi, Basis& out) {
  int n1 = t.p + 1;
  double v[MAXD][8], d[MAXD][8];
  for (int k = 0; k < dim; ++k) lagrange_eval(t.gll.data(), n1, xi[k], v[k], d[k]);
  int B = 1;
  for (int k = 0; k < dim; ++k) B *= n1;
  for (int i = 0; i < B; ++i) {
    int idx[MAXD];
    int r = i;
    for (int k = 0; k < dim; ++k) { idx[k] = r % n1; r /= n1; }
    double ph = 1.0;
    for (int k = 0; k < dim; ++k) ph *= v[k][idx[k]];
    out.phi[i] = ph;
    for (int l = 0; l < dim; ++l) {
      double gl = 1.0;
      for (int k = 0; k < dim; ++k) gl *= (k == l) ? d[k][idx[k]] : v[k][idx[k]];
      out.g[i][l] = gl;
    }
  }
}

}  // namespace

// multilinear map: x(xi) and J[k][l] = dx_k/dxi_l from the 2^dim corners
void map_point(int dim, const double* Xc, const double* xi, double* x, double J[MAXD][MAXD]) {
  int V = 1 << dim;
  for (int k = 0; k < dim; ++k) {
    x[k] = 0.0;
    for (int l = 0; l < dim; ++l) J[k][l] = 0.0;
  }
  for (int c = 0; c < V; ++c) {
    double N = 1.0;
    double dN[MAXD];
    for (int l = 0; l < dim; ++l) dN[l] = 1.0;
    for (int k = 0; k < dim; ++k) {
      int bit = (c >> k) & 1;
      double f = bit ? xi[k] : 1.0 - xi[k];
      double df = bit ? 1.0 : -1.0;
      N *= f;
      for (int l = 0; l < dim; ++l) dN[l] *= (l == k) ? df : f;
    }
    for (int k = 0; k < dim; ++k) {
      x[k] += N * Xc[c * dim + k];
      for (int l = 0; l < dim; ++l) J[k][l] += dN[l] * Xc[c * dim + k];
    }
  }
}

double det_inv(int dim, double J[MAXD][MAXD], double Ji[MAXD][MAXD]) {
  if (dim == 2) {
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det;
    Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det;
    Ji[1][1] = J[0][0] / det;
    return det;
  }
  double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  Ji[0][0] = c00 / det;
  Ji[1][0] = c01 / det;
  Ji[2][0] = c02 / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  return det;
}

namespace {

// physical gradient: component k = sum_l Jinv[l][k] * ghat_l
inline void phys_grad(int dim, const double Ji[MAXD][MAXD], const double* gh, double* g) {
  for (int k = 0; k < dim; ++k) {
    double s = 0.0;
    for (int l = 0; l < dim; ++l) s += Ji[l][k] * gh[l];
    g[k] = s;
  }
}

// corners of local face f = 2k + s, in face-corner order (lowest remaining axis fastest)
int face_corners(int dim, int f, int* out) {
  int k = f / 2, s = f % 2;
  int others[MAXD], no = 0;
  for (int a = 0; a < dim; ++a)
    if (a != k) others[no++] = a;
  int nvf = 1 << (dim - 1);
  for (int m = 0; m < nvf; ++m) {
    int c = s << k;
    for (int j = 0; j < no; ++j) c |= ((m >> j) & 1) << others[j];
    out[m] = c;
  }
  return nvf;
}

int axis_stride(int N, int a) { return a == 0 ? 1 : (a == 1 ? N : N * N); }
// r-th DoF on local face f (r = j1 + N j2 over the tangential axes in increasing order)
int face_dof(int dim, int N, int f, int r) {
  const int k = f / 2, s = f % 2;
  int t[2] = {0, 0}, no = 0;
  for (int a = 0; a < dim; ++a)
    if (a != k) t[no++] = a;
  int idx = s * (N - 1) * axis_stride(N, k) + (r % N) * axis_stride(N, t[0]);
  if (dim == 3) idx += (r / N) * axis_stride(N, t[1]);
  return idx;
}
// r-th DoF off local face f (r = j1 + N j2 + NF i', i' the normal index with
// the face layer left out)
int off_dof(int dim, int N, int f, int r) {
  const int k = f / 2, s = f % 2, NF = dim == 2 ? N : N * N;
  return (r / NF + 1 - s) * axis_stride(N, k) + face_dof(dim, N, 2 * k, r % NF);
}
}  // namespace

// ---------------------------------------------------------------- assembly
int mesh_build(Mesh& m, std::string& err) {
  const int dim = m.dim, p = m.p;
  if (dim != 2 && dim != 3) { err = "dim must be 2 or 3"; return AGG_EINVAL; }
  if (p < 1 || p > 4) { err = "degree must be in 1..4"; return AGG_EINVAL; }
  if (m.quad_extra < 0 || m.quad_extra > 4) { err = "quad_extra must be in 0..4"; return AGG_EINVAL; }
  const int n1 = p + 1;
  int B = 1;
  for (int k = 0; k < dim; ++k) B *= n1;
  m.B = B;
  const int V = 1 << dim;
  const int64_t ne = m.ne;
  for (int64_t i = 0; i < ne * V; ++i)
    if (m.cells[i] < 0 || m.cells[i] >= m.nv) { err = "vertex id out of range"; return AGG_EINVAL; }
  const double c_pen = (m.penalty_mode == 0) ? double(p * (p + 1)) : m.penalty_coeff * p * p;

  const int q = p + 1 + m.quad_extra;
  Tables1D t = make_tables(p, q);
  // volume quadrature: tensor Gauss points, x fastest
  int Q = 1;
  for (int k = 0; k < dim; ++k) Q *= q;
  std::vector<double> qx(Q * dim), qw(Q);
  for (int iq = 0; iq < Q; ++iq) {
    int r = iq;
    double w = 1.0;
    for (int k = 0; k < dim; ++k) {
      int a = r % q;
      r /= q;
      qx[iq * dim + k] = t.gx[a];
      w *= t.gw[a];
    }
    qw[iq] = w;
  }
  std::vector<Basis> qb(Q);
  for (int iq = 0; iq < Q; ++iq) tensor_basis(t, dim, &qx[iq * dim], qb[iq]);
  // face quadrature: tensor Gauss in dim-1 coordinates
  int Qf = 1;
  for (int k = 0; k < dim - 1; ++k) Qf *= q;
  std::vector<double> ft(Qf * MAXD), fw(Qf);
  for (int iq = 0; iq < Qf; ++iq) {
    int r = iq;
    double w = 1.0;
    for (int k = 0; k < dim - 1; ++k) {
      int a = r % q;
      r /= q;
      ft[iq * MAXD + k] = t.gx[a];
      w *= t.gw[a];
    }
    fw[iq] = w;
  }

  m.Me.assign((size_t)ne * B * B, 0.0);
  std::vector<double> Ke((size_t)ne * B * B, 0.0);
  const bool adj = m.adjoint_data;
  m.vol.assign(ne, 0.0);
  int bad_jac = 0;

#pragma omp parallel for schedule(static) reduction(+ : bad_jac)
  for (int64_t e = 0; e < ne; ++e) {
    double Xc[8 * MAXD];
    for (int c = 0; c < V; ++c)
      for (int k = 0; k < dim; ++k) Xc[c * dim + k] = m.X[m.cells[e * V + c] * dim + k];
    const double* De = &m.D[e * dim * dim];
    double* Mb = &m.Me[(size_t)e * B * B];
    double* Kb = &Ke[(size_t)e * B * B];
    double vol = 0.0;
    std::vector<double> G((size_t)B * MAXD), DG((size_t)B * MAXD);
    for (int iq = 0; iq < Q; ++iq) {
      double x[MAXD], J[MAXD][MAXD], Ji[MAXD][MAXD];
      map_point(dim, Xc, &qx[iq * dim], x, J);
      double det = det_inv(dim, J, Ji);
      if (!(det > 0.0)) { bad_jac += 1; continue; }
      double wJ = qw[iq] * det;
      vol += wJ;
      const Basis& b = qb[iq];
      for (int i = 0; i < B; ++i) {
        phys_grad(dim, Ji, b.g[i], &G[i * MAXD]);
        for (int k = 0; k < dim; ++k) {
          double s = 0.0;
          for (int l = 0; l < dim; ++l) s += De[k * dim + l] * G[i * MAXD + l];
          DG[i * MAXD + k] = s;
        }
      }
      for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) {
          Mb[i * B + j] += wJ * b.phi[i] * b.phi[j];
          double s = 0.0;
          for (int k = 0; k < dim; ++k) s += G[i * MAXD + k] * DG[j * MAXD + k];
          Kb[i * B + j] += wJ * s;
        }
    }
    m.vol[e] = vol;
  }
  if (bad_jac) { err = "element with non-positive Jacobian"; return AGG_EINVAL; }

  // ---------------- face matching by sorted vertex ids
  const int nf = 2 * dim;
  const int nvf = 1 << (dim - 1);
  int fcorn[6][4];
  for (int f = 0; f < nf; ++f) face_corners(dim, f, fcorn[f]);
  struct Key {
    std::array<int64_t, 4> v;
    int64_t rec;
  };
  std::vector<Key> keys((size_t)ne * nf);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ne; ++e)
    for (int f = 0; f < nf; ++f) {
      Key& k = keys[e * nf + f];
      k.v = {-1, -1, -1, -1};
      for (int mm = 0; mm < nvf; ++mm) k.v[mm] = m.cells[e * V + fcorn[f][mm]];
      std::sort(k.v.begin(), k.v.begin() + nvf);
      k.rec = e * nf + f;
    }
  std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
    if (a.v != b.v) return a.v < b.v;
    return a.rec < b.rec;
  });
  std::vector<int64_t> nbr((size_t)ne * nf, -1);   // neighbour record e'*nf + f'
  int64_t nint = 0;
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j].v == keys[i].v) ++j;
    if (j - i == 2) {
      nbr[keys[i].rec] = keys[i + 1].rec;
      nbr[keys[i + 1].rec] = keys[i].rec;
      ++nint;
    } else if (j - i > 2) {
      err = "a face is shared by more than two elements";
      return AGG_EINVAL;
    }
    i = j;
  }
  m.n_faces = nint;
  m.face_nbr = nbr;
  m.face_rev.assign((size_t)ne * nf, 0);
  for (int64_t e = 0; e < ne; ++e)
    for (int f = 0; f < nf; ++f) {
      const int64_t rec = nbr[e * nf + f];
      if (rec < 0) continue;
      const int64_t n = rec / nf;
      const int fn = (int)(rec % nf);
      m.face_rev[e * nf + f] = (int8_t)(m.cells[n * V + fcorn[fn][0]] != m.cells[e * V + fcorn[f][0]]);
    }

  // ---------------- block rows: diagonal + one block per interior face
  m.A.nrows = ne;
  m.A.B = B;
  m.A.rowptr.assign(ne + 1, 0);
  for (int64_t e = 0; e < ne; ++e) {
    int cnt = 1;
    for (int f = 0; f < nf; ++f) cnt += nbr[e * nf + f] >= 0;
    m.A.rowptr[e + 1] = m.A.rowptr[e] + cnt;
  }
  const int64_t nnzb = m.A.rowptr[ne];
  m.A.col.assign(nnzb, 0);
  m.A.val.assign((size_t)nnzb * B * B, 0.0);
  m.face_slot.assign((size_t)ne * nf, -1);
  const int NFd = (dim == 2) ? (m.p + 1) : (m.p + 1) * (m.p + 1);
  if (adj) m.Yc.assign((size_t)ne * nf * 4 * NFd * B, 0.0);
  int bad_face = 0;

#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad_face)
  for (int64_t e = 0; e < ne; ++e) {
    // column order: sorted neighbour ids (diagonal included)
    int64_t cols[7];
    int fof[7];
    int nc = 0;
    cols[nc] = e;
    fof[nc++] = -1;
    for (int f = 0; f < nf; ++f)
      if (nbr[e * nf + f] >= 0) {
        cols[nc] = nbr[e * nf + f] / nf;
        fof[nc++] = f;
      }
    int ord[7];
    for (int i = 0; i < nc; ++i) ord[i] = i;
    std::sort(ord, ord + nc, [&](int a, int b) { return cols[a] < cols[b]; });
    const int64_t base = m.A.rowptr[e];
    int diag_slot = -1;
    int slot_of[7];
    for (int s = 0; s < nc; ++s) {
      m.A.col[base + s] = (int32_t)cols[ord[s]];
      slot_of[ord[s]] = s;
      if (ord[s] == 0) diag_slot = s;
    }
    for (int i = 1; i < nc; ++i) m.face_slot[e * nf + fof[i]] = (int32_t)slot_of[i];
    double* Adiag = &m.A.val[(size_t)(base + diag_slot) * B * B];
    std::memcpy(Adiag, &Ke[(size_t)e * B * B], sizeof(double) * B * B);

    double Xp[8 * MAXD], Xm[8 * MAXD];
    for (int c = 0; c < V; ++c)
      for (int k = 0; k < dim; ++k) Xp[c * dim + k] = m.X[m.cells[e * V + c] * dim + k];
    const double* Dp = &m.D[e * dim * dim];
    std::vector<double> php(B), phm(B), flp(B), flm(B), sig(Qf), wdS(Qf);
    std::vector<double> PHP((size_t)Qf * B), PHM((size_t)Qf * B), FLP((size_t)Qf * B),
        FLM((size_t)Qf * B);
    for (int i = 1; i < nc; ++i) {
      const int f = fof[i];
      const int64_t rec = nbr[e * nf + f];
      const int64_t n = rec / nf;
      const int fn = (int)(rec % nf);
      for (int c = 0; c < V; ++c)
        for (int k = 0; k < dim; ++k) Xm[c * dim + k] = m.X[m.cells[n * V + c] * dim + k];
      const double* Dm = &m.D[n * dim * dim];
      // reference coordinates on the neighbour of each face corner of e
      double cxi[4][MAXD];
      for (int mm = 0; mm < nvf; ++mm) {
        int64_t gid = m.cells[e * V + fcorn[f][mm]];
        int found = -1;
        for (int mk = 0; mk < nvf; ++mk)
          if (m.cells[n * V + fcorn[fn][mk]] == gid) found = fcorn[fn][mk];
        if (found < 0) { bad_face += 1; found = 0; }
        for (int k = 0; k < dim; ++k) cxi[mm][k] = (found >> k) & 1;
      }
      const int kf = f / 2, sf = f % 2;
      int others[MAXD], no = 0;
      for (int a = 0; a < dim; ++a)
        if (a != kf) others[no++] = a;
      double area = 0.0;
      std::vector<std::array<double, MAXD>> nrm(Qf);
      for (int iq = 0; iq < Qf; ++iq) {
        const double* tq = &ft[iq * MAXD];
        double xip[MAXD], xim[MAXD];
        xip[kf] = sf;
        for (int j = 0; j < no; ++j) xip[others[j]] = tq[j];
        for (int k = 0; k < dim; ++k) xim[k] = 0.0;
        for (int mm = 0; mm < nvf; ++mm) {
          double Nf = 1.0;
          for (int j = 0; j < dim - 1; ++j) Nf *= ((mm >> j) & 1) ? tq[j] : 1.0 - tq[j];
          for (int k = 0; k < dim; ++k) xim[k] += Nf * cxi[mm][k];
        }
        // the neighbour's normal coordinate is constant on its face: set it
        // exactly, so that its basis functions with nodes off the face vanish
        // there exactly (the interpolated value is off by rounding)
        xim[fn / 2] = (double)(fn % 2);
        double xp[MAXD], xm[MAXD], Jp[MAXD][MAXD], Jm[MAXD][MAXD], Jip[MAXD][MAXD], Jim[MAXD][MAXD];
        map_point(dim, Xp, xip, xp, Jp);
        map_point(dim, Xm, xim, xm, Jm);
        double detp = det_inv(dim, Jp, Jip);
        det_inv(dim, Jm, Jim);
        double dist = 0.0, scale = 1.0;
        for (int k = 0; k < dim; ++k) {
          dist = std::max(dist, std::fabs(xp[k] - xm[k]));
          scale = std::max(scale, std::fabs(xp[k]));
        }
        if (dist > 1e-10 * scale) bad_face += 1;
        double nv[MAXD], len = 0.0;
        for (int k = 0; k < dim; ++k) {
          nv[k] = Jip[kf][k] * (2.0 * sf - 1.0);      // J^{-T} nhat
          len += nv[k] * nv[k];
        }
        len = std::sqrt(len);
        for (int k = 0; k < dim; ++k) nrm[iq][k] = nv[k] / len;
        wdS[iq] = fw[iq] * detp * len;
        area += wdS[iq];
        Basis bp, bm;
        tensor_basis(t, dim, xip, bp);
        tensor_basis(t, dim, xim, bm);
        for (int j = 0; j < B; ++j) {
          double gp[MAXD], gm[MAXD];
          phys_grad(dim, Jip, bp.g[j], gp);
          phys_grad(dim, Jim, bm.g[j], gm);
          double fp = 0.0, fm = 0.0;
          for (int k = 0; k < dim; ++k)
            for (int l = 0; l < dim; ++l) {
              fp += nrm[iq][k] * Dp[k * dim + l] * gp[l];
              fm += nrm[iq][k] * Dm[k * dim + l] * gm[l];
            }
          PHP[iq * B + j] = bp.phi[j];
          PHM[iq * B + j] = bm.phi[j];
          FLP[iq * B + j] = fp;
          FLM[iq * B + j] = fm;
        }
      }
      const double alpha = c_pen * std::max(area / m.vol[e], area / m.vol[n]);
      for (int iq = 0; iq < Qf; ++iq) {
        double s = 0.0;
        for (int k = 0; k < dim; ++k)
          for (int l = 0; l < dim; ++l) s += nrm[iq][k] * 0.5 * (Dp[k * dim + l] + Dm[k * dim + l]) * nrm[iq][l];
        sig[iq] = alpha * s;
      }
      double* Aoff = &m.A.val[(size_t)(base + slot_of[i]) * B * B];
      if (adj) {
        // part of this face's terms built with D_e (e on the + side): its
        // consistency terms and half of the penalty
        std::vector<double> sp(Qf);
        for (int iq = 0; iq < Qf; ++iq) {
          double s2 = 0.0;
          for (int k = 0; k < dim; ++k)
            for (int l = 0; l < dim; ++l) s2 += nrm[iq][k] * Dp[k * dim + l] * nrm[iq][l];
          sp[iq] = 0.5 * alpha * s2;
        }
        // only the entries a GLL nodal basis can make nonzero (a trace factor
        // vanishes off the face): ee on e's face rows / face columns, en on
        // n's face columns, ne on n's face rows, nn on both (layout in setup.h)
        auto yent = [&](int part, int a, int b) {
          double y = 0.0;
          for (int iq = 0; iq < Qf; ++iq) {
            const double w = wdS[iq], s2 = sp[iq];
            const double pa = PHP[iq * B + a], pb = PHP[iq * B + b];
            const double ma = PHM[iq * B + a], mb = PHM[iq * B + b];
            const double fa = FLP[iq * B + a], fb = FLP[iq * B + b];
            if (part == 0) y += w * (-0.5 * pa * fb - 0.5 * pb * fa + s2 * pa * pb);
            else if (part == 1) y += w * (0.5 * mb * fa - s2 * pa * mb);
            else if (part == 2) y += w * (0.5 * ma * fb - s2 * ma * pb);
            else y += w * (s2 * ma * mb);
          }
          return y;
        };
        const int NF = NFd, N1 = m.p + 1;
        double* Y = &m.Yc[((size_t)e * nf + f) * 4 * NF * B];
        double* yR = Y;                                  // NF x B
        double* yC = yR + NF * B;                        // (B - NF) x NF
        double* yEN = yC + (B - NF) * NF;                // B x NF
        double* yNE = yEN + B * NF;                      // NF x B
        double* yNN = yNE + NF * B;                      // NF x NF
        for (int r = 0; r < NF; ++r)
          for (int c = 0; c < B; ++c) yR[r * B + c] = yent(0, face_dof(dim, N1, f, r), c);
        for (int r = 0; r < B - NF; ++r)
          for (int c = 0; c < NF; ++c) yC[r * NF + c] = yent(0, off_dof(dim, N1, f, r), face_dof(dim, N1, f, c));
        for (int r = 0; r < B; ++r)
          for (int c = 0; c < NF; ++c) yEN[r * NF + c] = yent(1, r, face_dof(dim, N1, fn, c));
        for (int r = 0; r < NF; ++r)
          for (int c = 0; c < B; ++c) yNE[r * B + c] = yent(2, face_dof(dim, N1, fn, r), c);
        for (int r = 0; r < NF; ++r)
          for (int c = 0; c < NF; ++c) yNN[r * NF + c] = yent(3, face_dof(dim, N1, fn, r), face_dof(dim, N1, fn, c));
      }
      for (int a = 0; a < B; ++a)
        for (int b = 0; b < B; ++b) {
          double spp = 0.0, spm = 0.0;
          for (int iq = 0; iq < Qf; ++iq) {
            const double ia = PHP[iq * B + a], fa = FLP[iq * B + a];
            spp += wdS[iq] * (-0.5 * ia * FLP[iq * B + b] - 0.5 * PHP[iq * B + b] * fa +
                              sig[iq] * ia * PHP[iq * B + b]);
            spm += wdS[iq] * (-0.5 * ia * FLM[iq * B + b] + 0.5 * PHM[iq * B + b] * fa -
                              sig[iq] * ia * PHM[iq * B + b]);
          }
          Adiag[a * B + b] += spp;
          Aoff[a * B + b] = spm;
        }
    }
  }
  if (bad_face) { err = "non-conforming face (quadrature points do not coincide)"; return AGG_EINVAL; }
  if (adj) m.Ke.swap(Ke);
  return AGG_OK;
}

int mesh_locate(const Mesh& m, int64_t n, const double* pts, int64_t* elem, double* weights, std::string& err) {
  const int dim = m.dim, V = 1 << dim, n1 = m.p + 1, B = m.B;
  Tables1D t = make_tables(m.p, m.p + 2);
  std::vector<double> lo((size_t)m.ne * dim, 1e300), hi((size_t)m.ne * dim, -1e300);
  for (int64_t e = 0; e < m.ne; ++e)
    for (int c = 0; c < V; ++c)
      for (int k = 0; k < dim; ++k) {
        const double x = m.X[m.cells[e * V + c] * dim + k];
        lo[e * dim + k] = std::min(lo[e * dim + k], x);
        hi[e * dim + k] = std::max(hi[e * dim + k], x);
      }
  int missing = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : missing)
  for (int64_t s = 0; s < n; ++s) {
    const double* x = pts + s * dim;
    bool found = false;
    for (int64_t e = 0; e < m.ne && !found; ++e) {
      bool inside = true;
      for (int k = 0; k < dim; ++k)
        inside = inside && x[k] >= lo[e * dim + k] - 1e-12 && x[k] <= hi[e * dim + k] + 1e-12;
      if (!inside) continue;
      double Xc[8 * MAXD];
      for (int c = 0; c < V; ++c)
        for (int k = 0; k < dim; ++k) Xc[c * dim + k] = m.X[m.cells[e * V + c] * dim + k];
      double xi[MAXD] = {0.5, 0.5, 0.5};
      for (int it = 0; it < 50; ++it) {
        double xx[MAXD], J[MAXD][MAXD], Ji[MAXD][MAXD];
        map_point(dim, Xc, xi, xx, J);
        det_inv(dim, J, Ji);
        double mx = 0.0;
        for (int k = 0; k < dim; ++k) {
          double d = 0.0;
          for (int l = 0; l < dim; ++l) d += Ji[k][l] * (xx[l] - x[l]);
          xi[k] -= d;
          mx = std::max(mx, std::fabs(d));
        }
        if (mx < 1e-15) break;
      }
      bool in_ref = true;
      for (int k = 0; k < dim; ++k) in_ref = in_ref && xi[k] >= -1e-10 && xi[k] <= 1.0 + 1e-10;
      if (!in_ref) continue;
      for (int k = 0; k < dim; ++k) xi[k] = std::min(1.0, std::max(0.0, xi[k]));
      Basis b;
      tensor_basis(t, dim, xi, b);
      elem[s] = e;
      for (int i = 0; i < B; ++i) weights[s * B + i] = b.phi[i];
      found = true;
    }
    if (!found) missing += 1;
  }
  (void)n1;
  if (missing) { err = std::to_string(missing) + " point(s) outside the mesh"; return AGG_EINVAL; }
  return AGG_OK;
}

void bsr_apply(const BlockCSR& A, const double* x, double* y) {
  const int B = A.B;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < A.nrows; ++r) {
    double acc[MAXB];
    for (int i = 0; i < B; ++i) acc[i] = 0.0;
    for (int64_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      const double* blk = &A.val[(size_t)k * B * B];
      const double* xc = x + (int64_t)A.col[k] * B;
      for (int i = 0; i < B; ++i) {
        double s = 0.0;
        for (int j = 0; j < B; ++j) s += blk[i * B + j] * xc[j];
        acc[i] += s;
      }
    }
    for (int i = 0; i < B; ++i) y[r * B + i] = acc[i];
  }
}

}  // namespace aggmg

namespace aggmg {

static int matrix_free_build_3d(const Mesh& m, const std::vector<int64_t>& perm, const std::vector<int64_t>& inv,
                                double c, MatrixFreeData& out, std::string& err);

int matrix_free_build(const Mesh& m, const std::vector<int64_t>& perm, const std::vector<int64_t>& inv, double c,
                      MatrixFreeData& out, std::string& err) {
  if (m.dim == 3) return matrix_free_build_3d(m, perm, inv, c, out, err);
  if (m.dim != 2) { err = "the matrix-free fine operator is built for 2D and 3D meshes"; return AGG_EUNSUPPORTED; }
  const int dim = 2, V = 4, nf = 4, p = m.p;
  const int q = p + 1 + m.quad_extra;
  const int Q = q * q;
  const double c_pen = (m.penalty_mode == 0) ? double(p * (p + 1)) : m.penalty_coeff * p * p;
  Tables1D t = make_tables(p, q);
  const int64_t ne = m.ne;
  const int64_t nsl = (ne + 31) / 32;
  out.q = q;
  out.cell.assign((size_t)nsl * 32 * Q * 4, 0.0);
  out.face.assign((size_t)nsl * 32 * nf * q * 5, 0.0);
  out.nbr.assign((size_t)nsl * 32 * nf, -1);
  out.code.assign((size_t)nsl * 32 * nf, 0);
  int fcorn[4][2];
  for (int f = 0; f < nf; ++f) face_corners(dim, f, fcorn[f]);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t r = 0; r < ne; ++r) {
    const int64_t e = perm[r];
    const int64_t sl = r / 32, lane = r % 32;
    double Xe[8], Xn[8];
    for (int cc = 0; cc < V; ++cc)
      for (int k = 0; k < dim; ++k) Xe[cc * dim + k] = m.X[m.cells[e * V + cc] * dim + k];
    const double* De = &m.D[e * 4];
    // cell quadrature: G = w |J| J^-1 D J^-T, m = c w |J|
    for (int iq = 0; iq < Q; ++iq) {
      double xi[2] = {t.gx[iq % q], t.gx[iq / q]};
      const double w = t.gw[iq % q] * t.gw[iq / q];
      double x[2], J[MAXD][MAXD], Ji[MAXD][MAXD];
      map_point(dim, Xe, xi, x, J);
      const double det = det_inv(dim, J, Ji);
      if (!(det > 0)) bad += 1;
      double G[2][2];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          double sacc = 0.0;
          for (int k = 0; k < 2; ++k)
            for (int l = 0; l < 2; ++l) sacc += Ji[a][k] * De[k * 2 + l] * Ji[b][l];
          G[a][b] = w * det * sacc;
        }
      const double vals[4] = {G[0][0], G[0][1], G[1][1], c * w * det};
      for (int comp = 0; comp < 4; ++comp)
        out.cell[((size_t)sl * Q * 4 + iq * 4 + comp) * 32 + lane] = vals[comp];
    }
    // faces
    for (int f = 0; f < nf; ++f) {
      const int64_t rec = m.face_nbr[e * nf + f];
      if (rec < 0) continue;
      const int64_t n = rec / nf;
      const int fn = (int)(rec % nf);
      const int rev = m.face_rev[e * nf + f];
      out.nbr[((size_t)sl * nf + f) * 32 + lane] = (int32_t)inv[n];
      out.code[((size_t)sl * nf + f) * 32 + lane] = (int8_t)(fn * 2 + rev);
      for (int cc = 0; cc < V; ++cc)
        for (int k = 0; k < dim; ++k) Xn[cc * dim + k] = m.X[m.cells[n * V + cc] * dim + k];
      const double* Dn = &m.D[n * 4];
      const int kf = f / 2, sf = f % 2, kn = fn / 2, sn = fn % 2;
      double area = 0.0;
      std::vector<double> a0(q), a1(q), b0(q), b1(q), sg(q), wdS(q);
      for (int iq = 0; iq < q; ++iq) {
        const double tq = t.gx[iq];
        double xip[2], xim[2];
        xip[kf] = sf;
        xip[1 - kf] = tq;
        xim[kn] = sn;
        xim[1 - kn] = rev ? 1.0 - tq : tq;
        double xp[2], xm[2], Jp[MAXD][MAXD], Jm[MAXD][MAXD], Jip[MAXD][MAXD], Jim[MAXD][MAXD];
        map_point(dim, Xe, xip, xp, Jp);
        map_point(dim, Xn, xim, xm, Jm);
        const double detp = det_inv(dim, Jp, Jip);
        det_inv(dim, Jm, Jim);
        if (std::fabs(xp[0] - xm[0]) + std::fabs(xp[1] - xm[1]) > 1e-10 * (1.0 + std::fabs(xp[0]) + std::fabs(xp[1])))
          bad += 1;
        double nv[2], len = 0.0;
        for (int k = 0; k < 2; ++k) {
          nv[k] = Jip[kf][k] * (2.0 * sf - 1.0);
          len += nv[k] * nv[k];
        }
        len = std::sqrt(len);
        const double nn[2] = {nv[0] / len, nv[1] / len};
        wdS[iq] = t.gw[iq] * detp * len;
        area += wdS[iq];
        double Den[2], Dnn[2];
        for (int k = 0; k < 2; ++k) {
          Den[k] = De[k * 2 + 0] * nn[0] + De[k * 2 + 1] * nn[1];
          Dnn[k] = Dn[k * 2 + 0] * nn[0] + Dn[k * 2 + 1] * nn[1];
        }
        // a = wdS J_e^-1 D_e n (reference-gradient coefficients), b likewise on the neighbour
        a0[iq] = wdS[iq] * (Jip[0][0] * Den[0] + Jip[0][1] * Den[1]);
        a1[iq] = wdS[iq] * (Jip[1][0] * Den[0] + Jip[1][1] * Den[1]);
        b0[iq] = wdS[iq] * (Jim[0][0] * Dnn[0] + Jim[0][1] * Dnn[1]);
        b1[iq] = wdS[iq] * (Jim[1][0] * Dnn[0] + Jim[1][1] * Dnn[1]);
        double nDn = 0.0;
        for (int k = 0; k < 2; ++k)
          for (int l = 0; l < 2; ++l) nDn += nn[k] * 0.5 * (De[k * 2 + l] + Dn[k * 2 + l]) * nn[l];
        sg[iq] = nDn;
      }
      const double alpha = c_pen * std::max(area / m.vol[e], area / m.vol[n]);
      for (int iq = 0; iq < q; ++iq) {
        const double vals[5] = {a0[iq], a1[iq], b0[iq], b1[iq], wdS[iq] * alpha * sg[iq]};
        for (int comp = 0; comp < 5; ++comp)
          out.face[(((size_t)sl * nf + f) * q * 5 + iq * 5 + comp) * 32 + lane] = vals[comp];
      }
    }
  }
  if (bad) { err = "matrix-free geometry: bad Jacobian or non-matching face points"; return AGG_EINVAL; }
  return AGG_OK;
}


// 3D: cell[slice][qp*7 + {G00, G01, G02, G11, G12, G22, m}][lane] at Q^3 points
// (qp = k + Q l + Q^2 m'), face[slice][f][q*7 + {aN, aT0, aT1, bN, bT0, bT1, s}][lane]
// at Q^2 points per face (q = q1 + Q q2 along the face's remaining axes in
// increasing order; a and b in their side's face frame), code = neighbour's
// local face. The neighbour's face must be parametrised the same way (matching
// face-corner order); otherwise the matrix-free operator is unsupported.
static int matrix_free_build_3d(const Mesh& m, const std::vector<int64_t>& perm, const std::vector<int64_t>& inv,
                                double c, MatrixFreeData& out, std::string& err) {
  const int dim = 3, V = 8, nf = 6, p = m.p;
  const int q = p + 1 + m.quad_extra;
  const int Q3 = q * q * q, Q2 = q * q;
  const double c_pen = (m.penalty_mode == 0) ? double(p * (p + 1)) : m.penalty_coeff * p * p;
  Tables1D t = make_tables(p, q);
  const int64_t ne = m.ne;
  const int64_t nsl = (ne + 31) / 32;
  out.q = q;
  out.cell.assign((size_t)nsl * 32 * Q3 * 7, 0.0);
  out.face.assign((size_t)nsl * 32 * nf * Q2 * 7, 0.0);
  out.nbr.assign((size_t)nsl * 32 * nf, -1);
  out.code.assign((size_t)nsl * 32 * nf, 0);
  int fcorn[6][4];
  for (int f = 0; f < nf; ++f) face_corners(dim, f, fcorn[f]);
  int bad = 0, misoriented = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad, misoriented)
  for (int64_t r = 0; r < ne; ++r) {
    const int64_t e = perm[r];
    const int64_t sl = r / 32, lane = r % 32;
    double Xe[8 * MAXD], Xn[8 * MAXD];
    for (int cc = 0; cc < V; ++cc)
      for (int k = 0; k < dim; ++k) Xe[cc * dim + k] = m.X[m.cells[e * V + cc] * dim + k];
    const double* De = &m.D[e * 9];
    for (int iq = 0; iq < Q3; ++iq) {
      double xi[3] = {t.gx[iq % q], t.gx[(iq / q) % q], t.gx[iq / Q2]};
      const double w = t.gw[iq % q] * t.gw[(iq / q) % q] * t.gw[iq / Q2];
      double x[3], J[MAXD][MAXD], Ji[MAXD][MAXD];
      map_point(dim, Xe, xi, x, J);
      const double det = det_inv(dim, J, Ji);
      if (!(det > 0)) bad += 1;
      double G[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double sacc = 0.0;
          for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) sacc += Ji[a][k] * De[k * 3 + l] * Ji[b][l];
          G[a][b] = w * det * sacc;
        }
      const double vals[7] = {G[0][0], G[0][1], G[0][2], G[1][1], G[1][2], G[2][2], c * w * det};
      for (int comp = 0; comp < 7; ++comp)
        out.cell[((size_t)sl * Q3 * 7 + iq * 7 + comp) * 32 + lane] = vals[comp];
    }
    for (int f = 0; f < nf; ++f) {
      const int64_t rec = m.face_nbr[e * nf + f];
      if (rec < 0) continue;
      const int64_t n = rec / nf;
      const int fn = (int)(rec % nf);
      bool same = true;
      for (int mm = 0; mm < 4; ++mm) same = same && (m.cells[n * V + fcorn[fn][mm]] == m.cells[e * V + fcorn[f][mm]]);
      if (!same) {
        misoriented += 1;
        continue;
      }
      out.nbr[((size_t)sl * nf + f) * 32 + lane] = (int32_t)inv[n];
      out.code[((size_t)sl * nf + f) * 32 + lane] = (int8_t)fn;
      for (int cc = 0; cc < V; ++cc)
        for (int k = 0; k < dim; ++k) Xn[cc * dim + k] = m.X[m.cells[n * V + cc] * dim + k];
      const double* Dn = &m.D[n * 9];
      const int kf = f / 2, sf = f % 2, kn = fn / 2, sn = fn % 2;
      int oe[2], on[2], no = 0, nn = 0;
      for (int a = 0; a < 3; ++a) {
        if (a != kf) oe[no++] = a;
        if (a != kn) on[nn++] = a;
      }
      double area = 0.0;
      std::vector<double> av(Q2 * 3), bv(Q2 * 3), sg(Q2), wdS(Q2);
      for (int iq = 0; iq < Q2; ++iq) {
        const double t1 = t.gx[iq % q], t2 = t.gx[iq / q];
        double xip[3], xim[3];
        xip[kf] = sf;
        xip[oe[0]] = t1;
        xip[oe[1]] = t2;
        xim[kn] = sn;
        xim[on[0]] = t1;
        xim[on[1]] = t2;
        double xp[3], xm[3], Jp[MAXD][MAXD], Jm[MAXD][MAXD], Jip[MAXD][MAXD], Jim[MAXD][MAXD];
        map_point(dim, Xe, xip, xp, Jp);
        map_point(dim, Xn, xim, xm, Jm);
        const double detp = det_inv(dim, Jp, Jip);
        det_inv(dim, Jm, Jim);
        double dist = 0.0, scale = 1.0;
        for (int k = 0; k < 3; ++k) {
          dist = std::max(dist, std::fabs(xp[k] - xm[k]));
          scale = std::max(scale, std::fabs(xp[k]));
        }
        if (dist > 1e-10 * scale) bad += 1;
        double nv[3], len = 0.0;
        for (int k = 0; k < 3; ++k) {
          nv[k] = Jip[kf][k] * (2.0 * sf - 1.0);
          len += nv[k] * nv[k];
        }
        len = std::sqrt(len);
        const double nu[3] = {nv[0] / len, nv[1] / len, nv[2] / len};
        wdS[iq] = t.gw[iq % q] * t.gw[iq / q] * detp * len;
        area += wdS[iq];
        double Den[3], Dnn[3];
        for (int k = 0; k < 3; ++k) {
          Den[k] = De[k * 3 + 0] * nu[0] + De[k * 3 + 1] * nu[1] + De[k * 3 + 2] * nu[2];
          Dnn[k] = Dn[k * 3 + 0] * nu[0] + Dn[k * 3 + 1] * nu[1] + Dn[k * 3 + 2] * nu[2];
        }
        // a and b in their side's face frame (normal axis, then the two tangential
        // axes in increasing order)
        const int eframe[3] = {kf, oe[0], oe[1]}, nframe[3] = {kn, on[0], on[1]};
        for (int a = 0; a < 3; ++a) {
          const int ae = eframe[a];
          av[iq * 3 + a] = wdS[iq] * (Jip[ae][0] * Den[0] + Jip[ae][1] * Den[1] + Jip[ae][2] * Den[2]);
          const int an = nframe[a];
          bv[iq * 3 + a] = wdS[iq] * (Jim[an][0] * Dnn[0] + Jim[an][1] * Dnn[1] + Jim[an][2] * Dnn[2]);
        }
        double nDn = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) nDn += nu[k] * 0.5 * (De[k * 3 + l] + Dn[k * 3 + l]) * nu[l];
        sg[iq] = nDn;
      }
      const double alpha = c_pen * std::max(area / m.vol[e], area / m.vol[n]);
      for (int iq = 0; iq < Q2; ++iq) {
        const double vals[7] = {av[iq * 3], av[iq * 3 + 1], av[iq * 3 + 2], bv[iq * 3], bv[iq * 3 + 1],
                                bv[iq * 3 + 2], wdS[iq] * alpha * sg[iq]};
        for (int comp = 0; comp < 7; ++comp)
          out.face[(((size_t)sl * nf + f) * Q2 * 7 + iq * 7 + comp) * 32 + lane] = vals[comp];
      }
    }
  }
  if (bad) { err = "matrix-free geometry: bad Jacobian or non-matching face points"; return AGG_EINVAL; }
  if (misoriented) {
    err = "matrix-free operator (3D) needs neighbours that parametrise shared faces alike";
    return AGG_EUNSUPPORTED;
  }
  return AGG_OK;
}




int face_blocks_build(const Mesh& m, const HostLevel& l0, FaceBlocks& out, std::string& err) {
  const int dim = m.dim, B = m.B, N = m.p + 1, nf = 2 * dim;
  const int NF = dim == 2 ? N : N * N;
  const int64_t n = m.ne;
  out.NF = NF;
  out.nf = nf;
  out.diag.assign((size_t)n * B * B, 0.0);
  out.R.assign((size_t)n * nf * NF * B, 0.0);
  out.C.assign((size_t)n * nf * (B - NF) * NF, 0.0);
  out.nbr.assign((size_t)n * nf, -1);
  out.code.assign((size_t)n * nf, 0);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t u = 0; u < n; ++u) {
    const int64_t e = l0.perm[u];
    bool found = false;
    for (int64_t j = l0.A.rowptr[u]; j < l0.A.rowptr[u + 1]; ++j)
      if (l0.A.col[j] == u) {
        std::memcpy(&out.diag[(size_t)u * B * B], &l0.A.val[(size_t)j * B * B], sizeof(double) * B * B);
        found = true;
      }
    if (!found) bad += 1;
    std::vector<char> on_fn(B);
    for (int f = 0; f < nf; ++f) {
      const int64_t rec = m.face_nbr[e * nf + f];
      if (rec < 0) continue;
      const int64_t nb = rec / nf;
      const int fn = (int)(rec % nf);
      out.nbr[u * nf + f] = (int32_t)l0.inv[nb];
      out.code[u * nf + f] = (int8_t)fn;
      const double* blk = &m.A.val[(size_t)(m.A.rowptr[e] + m.face_slot[e * nf + f]) * B * B];
      double* R = &out.R[((size_t)u * nf + f) * NF * B];
      double* C = &out.C[((size_t)u * nf + f) * (B - NF) * NF];
      for (int r = 0; r < NF; ++r)
        for (int c = 0; c < B; ++c) R[r * B + c] = blk[face_dof(dim, N, f, r) * B + c];
      std::fill(on_fn.begin(), on_fn.end(), 0);
      for (int jf = 0; jf < NF; ++jf) on_fn[face_dof(dim, N, fn, jf)] = 1;
      for (int r = 0; r < B - NF; ++r) {
        const int row = off_dof(dim, N, f, r);
        for (int jf = 0; jf < NF; ++jf) C[r * NF + jf] = blk[row * B + face_dof(dim, N, fn, jf)];
        for (int c = 0; c < B; ++c)
          if (!on_fn[c] && blk[row * B + c] != 0.0) bad += 1;
      }
    }
  }
  if (bad) {
    err = "the fine operator lacks the face structure of a GLL nodal basis";
    return AGG_EINVAL;
  }
  return AGG_OK;
}


void adjoint_face_parts_full(const Mesh& m, double* out) {
  const int dim = m.dim, B = m.B, N = m.p + 1, nf = 2 * dim;
  const int NF = dim == 2 ? N : N * N;
  std::fill(out, out + (size_t)m.A.nnzb() * 4 * B * B, 0.0);
  for (int64_t e = 0; e < m.ne; ++e)
    for (int f = 0; f < nf; ++f) {
      const int64_t rec = m.face_nbr[e * nf + f];
      if (rec < 0) continue;
      const int fn = (int)(rec % nf);
      const double* Y = &m.Yc[((size_t)e * nf + f) * 4 * NF * B];
      const double *yR = Y, *yC = yR + NF * B, *yEN = yC + (B - NF) * NF, *yNE = yEN + B * NF,
                   *yNN = yNE + NF * B;
      double* o = out + (size_t)(m.A.rowptr[e] + m.face_slot[e * nf + f]) * 4 * B * B;
      double *ee = o, *en = o + B * B, *nee = o + 2 * B * B, *nn = o + 3 * B * B;
      for (int r = 0; r < NF; ++r)
        for (int c = 0; c < B; ++c) ee[face_dof(dim, N, f, r) * B + c] = yR[r * B + c];
      for (int r = 0; r < B - NF; ++r)
        for (int c = 0; c < NF; ++c) ee[off_dof(dim, N, f, r) * B + face_dof(dim, N, f, c)] = yC[r * NF + c];
      for (int r = 0; r < B; ++r)
        for (int c = 0; c < NF; ++c) en[r * B + face_dof(dim, N, fn, c)] = yEN[r * NF + c];
      for (int r = 0; r < NF; ++r)
        for (int c = 0; c < B; ++c) nee[face_dof(dim, N, fn, r) * B + c] = yNE[r * B + c];
      for (int r = 0; r < NF; ++r)
        for (int c = 0; c < NF; ++c) nn[face_dof(dim, N, fn, r) * B + face_dof(dim, N, fn, c)] = yNN[r * NF + c];
    }
}

}  // namespace aggmg
