// Non-inherited coarse operators (Section 5.1): the SIPG form with the mass
// term, c M_l + A_l, assembled directly on the agglomerates of level l >= 1
// by quadrature over the original mesh, with the level's Q_p box basis:
//   volume:  sum over the fine elements e of K of
//            int_e (grad phi_i^K)^T D_e grad phi_j^K + c phi_i^K phi_j^K;
//   faces:   every fine interior face between elements of different
//            agglomerates K+ (the side of the lower element id) and K-:
//            -1/2 sgn_i phi_i (D_sj grad phi_j . n) - 1/2 sgn_j phi_j (D_si grad phi_i . n)
//            + sigma sgn_i sgn_j phi_i phi_j,  n = the K+ element's outward normal,
//            sigma = C_pen max(|F_KK'|/|K|, |F_KK'|/|K'|) n^T ((D+ + D-)/2) n,
//            |F_KK'| = the measure of all fine faces between K and K'.
// The alternative to the inherited (Galerkin) operators that the paper uses;
// hierarchy_build takes it when HierOptions::direct is set.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/aggmg.h"
#include "setup.h"

namespace aggmg {

namespace {

constexpr int MAXD = 3;    // largest dimension

// Values and physical gradients of the Q_p box basis of [lo, hi] at x.
void box_basis(int dim, int p, const double* gll, const double* lo, const double* hi, const double* x, double* phi,
               double* grad /* [B][dim] */) {
  const int n1 = p + 1;
  double v[MAXD][8], d[MAXD][8];
  for (int k = 0; k < dim; ++k) {
    const double L = hi[k] - lo[k];
    lagrange_eval(gll, n1, (x[k] - lo[k]) / L, v[k], d[k]);
    for (int a = 0; a < n1; ++a) d[k][a] /= L;
  }
  int B = 1;
  for (int k = 0; k < dim; ++k) B *= n1;
  for (int j = 0; j < B; ++j) {
    int idx[MAXD], r = j;
    for (int k = 0; k < dim; ++k) {
      idx[k] = r % n1;
      r /= n1;
    }
    double val = 1.0;
    for (int k = 0; k < dim; ++k) val *= v[k][idx[k]];
    phi[j] = val;
    for (int k = 0; k < dim; ++k) {
      double g = 1.0;
      for (int kk = 0; kk < dim; ++kk) g *= (kk == k) ? d[kk][idx[kk]] : v[kk][idx[kk]];
      grad[j * dim + k] = g;
    }
  }
}

struct FacePoint {
  double x[MAXD], n[MAXD], wdS;
};

// Quadrature of local face f of element e: physical points, e's outward unit
// normal, weights times the surface measure.
void face_quadrature(const Mesh& m, int64_t e, int f, const std::vector<double>& ft, const std::vector<double>& fw,
                     std::vector<FacePoint>& out) {
  const int dim = m.dim, V = 1 << dim, Qf = (int)fw.size();
  const int kf = f / 2, sf = f % 2;
  int others[MAXD], no = 0;
  for (int a = 0; a < dim; ++a)
    if (a != kf) others[no++] = a;
  double X[8 * MAXD];
  for (int c = 0; c < V; ++c)
    for (int k = 0; k < dim; ++k) X[c * dim + k] = m.X[m.cells[e * V + c] * dim + k];
  out.resize(Qf);
  for (int iq = 0; iq < Qf; ++iq) {
    double xi[MAXD];
    xi[kf] = sf;
    for (int j = 0; j < no; ++j) xi[others[j]] = ft[iq * MAXD + j];
    double J[MAXD][MAXD], Ji[MAXD][MAXD];
    map_point(dim, X, xi, out[iq].x, J);
    const double det = det_inv(dim, J, Ji);
    double nv[MAXD], len = 0.0;
    for (int k = 0; k < dim; ++k) {
      nv[k] = Ji[kf][k] * (2.0 * sf - 1.0);
      len += nv[k] * nv[k];
    }
    len = std::sqrt(len);
    for (int k = 0; k < dim; ++k) out[iq].n[k] = nv[k] / len;
    out[iq].wdS = fw[iq] * det * len;
  }
}

}  // namespace

int direct_level_build(const Mesh& m, const HostHierarchy& h, int l, double c, BlockCSR& out, std::string& err) {
  const int dim = m.dim, p = m.p, B = m.B, nf = 2 * dim, V = 1 << dim, dd = dim * dim;
  const int q = p + 1 + m.quad_extra;
  const double c_pen = (m.penalty_mode == 0) ? double(p * (p + 1)) : m.penalty_coeff * p * p;
  const HostLevel& lv = h.lev[l];
  const int64_t nK = lv.n, ne = m.ne;
  // fine element -> unit of level l (internal order)
  std::vector<int64_t> unit(ne);
  for (int64_t e = 0; e < ne; ++e) {
    int64_t u = h.lev[0].inv[e];
    for (int k = 0; k < l; ++k) u = h.lev[k].parent[u];
    unit[e] = u;
  }
  std::vector<int64_t> eptr(nK + 1, 0), elist(ne);
  for (int64_t e = 0; e < ne; ++e) eptr[unit[e] + 1] += 1;
  for (int64_t K = 0; K < nK; ++K) eptr[K + 1] += eptr[K];
  {
    std::vector<int64_t> fill(eptr.begin(), eptr.end() - 1);
    for (int64_t e = 0; e < ne; ++e) elist[fill[unit[e]]++] = e;
  }
  // quadrature rules
  Tables1D t = make_tables(p, q);
  const int Q = (int)std::pow(q, dim);
  int Qf = 1;
  for (int k = 0; k < dim - 1; ++k) Qf *= q;
  std::vector<double> ft((size_t)Qf * MAXD, 0.0), fw(Qf);
  for (int iq = 0; iq < Qf; ++iq) {
    int r = iq;
    double w = 1.0;
    for (int k = 0; k < dim - 1; ++k) {
      const int a = r % q;
      r /= q;
      ft[iq * MAXD + k] = t.gx[a];
      w *= t.gw[a];
    }
    fw[iq] = w;
  }
  // agglomerate measures (volume quadrature) and polytopic face measures
  std::vector<double> volK(nK, 0.0);
  for (int64_t e = 0; e < ne; ++e) {
    double X[8 * MAXD];
    for (int cc = 0; cc < V; ++cc)
      for (int k = 0; k < dim; ++k) X[cc * dim + k] = m.X[m.cells[e * V + cc] * dim + k];
    double s = 0.0;
    for (int iq = 0; iq < Q; ++iq) {
      double xi[MAXD], w = 1.0, x[MAXD], J[MAXD][MAXD], Ji[MAXD][MAXD];
      int r = iq;
      for (int k = 0; k < dim; ++k) {
        xi[k] = t.gx[r % q];
        w *= t.gw[r % q];
        r /= q;
      }
      map_point(dim, X, xi, x, J);
      s += w * det_inv(dim, J, Ji);
    }
    volK[unit[e]] += s;
  }
  std::map<std::pair<int64_t, int64_t>, double> area;
  {
    std::vector<FacePoint> fq;
    for (int64_t e = 0; e < ne; ++e)
      for (int f = 0; f < nf; ++f) {
        const int64_t nb = m.face_nbr[e * nf + f];
        if (nb < 0) continue;
        const int64_t n = nb / nf;
        if (n < e || unit[n] == unit[e]) continue;          // each face once, from its lower element
        face_quadrature(m, e, f, ft, fw, fq);
        double s = 0.0;
        for (int iq = 0; iq < Qf; ++iq) s += fq[iq].wdS;
        const int64_t a = std::min(unit[e], unit[n]), b = std::max(unit[e], unit[n]);
        area[{a, b}] += s;
      }
  }
  // block rows, one agglomerate per iteration
  std::vector<std::vector<int32_t>> rcols(nK);
  std::vector<std::vector<double>> rvals(nK);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : bad)
  for (int64_t K = 0; K < nK; ++K) {
    std::vector<int32_t> cols{(int32_t)K};
    std::vector<double> acc((size_t)B * B, 0.0);
    std::vector<double> phs(B), gs((size_t)B * dim), pho(B), go((size_t)B * dim), fls(B), flo(B);
    std::vector<FacePoint> fq;
    const double* loK = &lv.lo[K * dim];
    const double* hiK = &lv.hi[K * dim];
    for (int64_t k = eptr[K]; k < eptr[K + 1]; ++k) {
      const int64_t e = elist[k];
      const double* De = &m.D[(size_t)e * dd];
      double X[8 * MAXD];
      for (int cc = 0; cc < V; ++cc)
        for (int kk = 0; kk < dim; ++kk) X[cc * dim + kk] = m.X[m.cells[e * V + cc] * dim + kk];
      // volume terms
      for (int iq = 0; iq < Q; ++iq) {
        double xi[MAXD], w = 1.0, x[MAXD], J[MAXD][MAXD], Ji[MAXD][MAXD];
        int r = iq;
        for (int kk = 0; kk < dim; ++kk) {
          xi[kk] = t.gx[r % q];
          w *= t.gw[r % q];
          r /= q;
        }
        map_point(dim, X, xi, x, J);
        const double det = det_inv(dim, J, Ji);
        if (!(det > 0)) bad += 1;
        const double wJ = w * det;
        box_basis(dim, p, t.gll.data(), loK, hiK, x, phs.data(), gs.data());
        for (int j = 0; j < B; ++j) {
          double Dg[MAXD];
          for (int a = 0; a < dim; ++a) {
            double s = 0.0;
            for (int b = 0; b < dim; ++b) s += De[a * dim + b] * gs[j * dim + b];
            Dg[a] = s;
          }
          for (int i = 0; i < B; ++i) {
            double s = 0.0;
            for (int a = 0; a < dim; ++a) s += gs[i * dim + a] * Dg[a];
            acc[(size_t)i * B + j] += wJ * (s + c * phs[i] * phs[j]);
          }
        }
      }
      // face terms of e's faces towards other agglomerates (this row's side)
      for (int f = 0; f < nf; ++f) {
        const int64_t nb = m.face_nbr[e * nf + f];
        if (nb < 0) continue;
        const int64_t n = nb / nf;
        const int fn = (int)(nb % nf);
        const int64_t Kn = unit[n];
        if (Kn == K) continue;
        const bool row_plus = e < n;                         // the lower element id is the + side
        face_quadrature(m, row_plus ? e : n, row_plus ? f : fn, ft, fw, fq);
        const double sgs = row_plus ? 1.0 : -1.0, sgo = -sgs;
        const auto it = area.find({std::min(K, Kn), std::max(K, Kn)});   // read-only here
        if (it == area.end()) {                                // a face the pair scan missed
          bad += 1;
          continue;
        }
        const double ar = it->second;
        const double alpha = c_pen * std::max(ar / volK[K], ar / volK[Kn]);
        const double* Dn = &m.D[(size_t)n * dd];
        size_t slot = 0;
        while (slot < cols.size() && cols[slot] != (int32_t)Kn) ++slot;
        if (slot == cols.size()) {
          cols.push_back((int32_t)Kn);
          acc.resize(acc.size() + (size_t)B * B, 0.0);
        }
        double* Ass = &acc[0];
        double* Aso = &acc[slot * (size_t)B * B];
        for (int iq = 0; iq < Qf; ++iq) {
          const FacePoint& P = fq[iq];
          box_basis(dim, p, t.gll.data(), loK, hiK, P.x, phs.data(), gs.data());
          box_basis(dim, p, t.gll.data(), &lv.lo[Kn * dim], &lv.hi[Kn * dim], P.x, pho.data(), go.data());
          double Den[MAXD], Dnn[MAXD], sig = 0.0;
          for (int a = 0; a < dim; ++a) {
            double s1 = 0.0, s2 = 0.0;
            for (int b = 0; b < dim; ++b) {
              s1 += De[a * dim + b] * P.n[b];
              s2 += Dn[a * dim + b] * P.n[b];
            }
            Den[a] = s1;
            Dnn[a] = s2;
          }
          for (int a = 0; a < dim; ++a) sig += P.n[a] * 0.5 * (Den[a] + Dnn[a]);
          sig *= alpha;
          for (int j = 0; j < B; ++j) {
            double s1 = 0.0, s2 = 0.0;
            for (int a = 0; a < dim; ++a) {
              s1 += gs[j * dim + a] * Den[a];
              s2 += go[j * dim + a] * Dnn[a];
            }
            fls[j] = s1;
            flo[j] = s2;
          }
          const double w = P.wdS;
          for (int i = 0; i < B; ++i)
            for (int j = 0; j < B; ++j) {
              Ass[(size_t)i * B + j] +=
                  w * (-0.5 * sgs * phs[i] * fls[j] - 0.5 * sgs * phs[j] * fls[i] + sig * phs[i] * phs[j]);
              Aso[(size_t)i * B + j] +=
                  w * (-0.5 * sgs * phs[i] * flo[j] - 0.5 * sgo * pho[j] * fls[i] + sgs * sgo * sig * phs[i] * pho[j]);
            }
        }
      }
    }
    std::vector<int> ord(cols.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return cols[a] < cols[b]; });
    rcols[K].resize(cols.size());
    rvals[K].resize(acc.size());
    for (size_t s = 0; s < ord.size(); ++s) {
      rcols[K][s] = cols[ord[s]];
      std::memcpy(&rvals[K][s * B * B], &acc[(size_t)ord[s] * B * B], sizeof(double) * B * B);
    }
  }
  if (bad) {
    err = "non-inherited coarse operator: non-positive Jacobian or an unmatched face";
    return AGG_EINVAL;
  }
  out.nrows = nK;
  out.B = B;
  out.rowptr.assign(nK + 1, 0);
  for (int64_t K = 0; K < nK; ++K) out.rowptr[K + 1] = out.rowptr[K] + (int64_t)rcols[K].size();
  out.col.resize(out.rowptr[nK]);
  out.val.resize((size_t)out.rowptr[nK] * B * B);
  for (int64_t K = 0; K < nK; ++K) {
    std::copy(rcols[K].begin(), rcols[K].end(), out.col.begin() + out.rowptr[K]);
    std::copy(rvals[K].begin(), rvals[K].end(), out.val.begin() + out.rowptr[K] * B * B);
  }
  return AGG_OK;
}

}  // namespace aggmg
