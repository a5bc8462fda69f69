// Host float64 set-up of the agglomerated hierarchy (Algorithm 3 and
// Section 5.1 of arXiv 2602.16312): unit orderings, bounding boxes,
// prolongation blocks, inherited Galerkin operators A_{l+1} = P^T A_l P in
// block form, block-Jacobi inverses, Lanczos Chebyshev bounds and the
// inverse Cholesky factor of the coarsest operator.
//
// Internal ordering: the units of every level are renumbered so that the
// children of each coarser unit are contiguous (sorted by parent, then by the
// caller's id). Restriction then becomes a segmented sum and neighbouring
// units stay close in memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "setup.h"
#include "../../include/aggmg.h"

namespace aggmg {

namespace {

// dense Cholesky in place (lower, row-major n x n); false if not SPD
bool cholesky(double* a, int64_t n) {
  for (int64_t j = 0; j < n; ++j) {
    double d = a[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    a[j * n + j] = d;
#pragma omp parallel for schedule(static) if (n > 256)
    for (int64_t i = j + 1; i < n; ++i) {
      double s = a[i * n + j];
      for (int64_t k = 0; k < j; ++k) s -= a[i * n + k] * a[j * n + k];
      a[i * n + j] = s / d;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) a[i * n + j] = 0.0;
  return true;
}

// inverse of a lower-triangular matrix (row-major), column by column
void lower_inverse(const double* L, double* Li, int64_t n) {
  std::fill(Li, Li + n * n, 0.0);
#pragma omp parallel for schedule(dynamic, 16) if (n > 256)
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int64_t k = c; k < i; ++k) s -= L[i * n + k] * Li[k * n + c];
      Li[i * n + c] = s / L[i * n + i];
    }
  }
}

// largest eigenvalue of the symmetric tridiagonal (a, b) by Sturm bisection
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int k = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < k - 1 ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
      double bb = (i > 0) ? b[i - 1] * b[i - 1] : 0.0;
      d = a[i] - x - (i > 0 ? bb / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (count_below(mid) == k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// C = A * Bm (B x B, row-major)
inline void gemm(const double* A, const double* Bm, double* C, int B) {
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) {
      double s = 0.0;
      for (int k = 0; k < B; ++k) s += A[i * B + k] * Bm[k * B + j];
      C[i * B + j] = s;
    }
}
// C += A^T * Bm
inline void gemm_tn_acc(const double* A, const double* Bm, double* C, int B) {
  for (int k = 0; k < B; ++k)
    for (int i = 0; i < B; ++i) {
      const double a = A[k * B + i];
      for (int j = 0; j < B; ++j) C[i * B + j] += a * Bm[k * B + j];
    }
}

void block_apply_host(const std::vector<double>& blocks, int B, const double* x, double* y, int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t u = 0; u < n; ++u)
    for (int i = 0; i < B; ++i) {
      double s = 0.0;
      for (int j = 0; j < B; ++j) s += blocks[((size_t)u * B + i) * B + j] * x[u * B + j];
      y[u * B + i] = s;
    }
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

}  // namespace

bool spd_inverse_blocks(const double* blocks, int64_t n, int B, double* out) {
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t u = 0; u < n; ++u) {
    std::vector<double> Lc(blocks + (size_t)u * B * B, blocks + (size_t)(u + 1) * B * B), Li((size_t)B * B);
    if (!cholesky(Lc.data(), B)) { bad += 1; continue; }
    lower_inverse(Lc.data(), Li.data(), B);
    double* Di = out + (size_t)u * B * B;
    for (int i = 0; i < B; ++i)
      for (int j = 0; j < B; ++j) {
        double sacc = 0.0;
        for (int k = std::max(i, j); k < B; ++k) sacc += Li[k * B + i] * Li[k * B + j];
        Di[i * B + j] = sacc;
      }
  }
  return bad == 0;
}

int hierarchy_build(const Mesh& m, double c, const HierOptions& o, HostHierarchy& h, std::string& err) {
  const int L = o.L, B = m.B, dim = m.dim, p = m.p;
  if (L < 1) { err = "n_levels must be >= 1"; return AGG_EINVAL; }
  if (L > 1 && !o.maps) { err = "agglomeration maps missing"; return AGG_EINVAL; }
  h.L = L;
  h.B = B;
  h.dim = dim;
  h.p = p;
  h.mass_coeff = c;
  h.lev.assign(L, HostLevel());
  // ---- sizes and validation of the maps
  h.lev[0].n = m.ne;
  for (int l = 0; l + 1 < L; ++l) {
    const int32_t* mp = o.maps[l];
    if (!mp) { err = "agglomeration map is NULL"; return AGG_EINVAL; }
    int64_t nl = h.lev[l].n, nmax = -1;
    for (int64_t u = 0; u < nl; ++u) {
      if (mp[u] < 0) { err = "negative agglomerate id"; return AGG_EINVAL; }
      nmax = std::max<int64_t>(nmax, mp[u]);
    }
    std::vector<char> used(nmax + 1, 0);
    for (int64_t u = 0; u < nl; ++u) used[mp[u]] = 1;
    for (int64_t k = 0; k <= nmax; ++k)
      if (!used[k]) { err = "agglomerate ids are not contiguous (an id is unused)"; return AGG_EINVAL; }
    h.lev[l + 1].n = nmax + 1;
  }
  // ---- internal orderings (coarsest keeps the caller's order)
  {
    HostLevel& lc = h.lev[L - 1];
    lc.perm.resize(lc.n);
    lc.inv.resize(lc.n);
    std::iota(lc.perm.begin(), lc.perm.end(), 0);
    std::iota(lc.inv.begin(), lc.inv.end(), 0);
  }
  for (int l = L - 2; l >= 0; --l) {
    HostLevel& lf = h.lev[l];
    HostLevel& lc = h.lev[l + 1];
    const int32_t* mp = o.maps[l];
    std::vector<int64_t> key(lf.n);
    for (int64_t u = 0; u < lf.n; ++u) key[u] = lc.inv[mp[u]];
    lf.perm.resize(lf.n);
    std::iota(lf.perm.begin(), lf.perm.end(), 0);
    std::stable_sort(lf.perm.begin(), lf.perm.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    lf.inv.resize(lf.n);
    for (int64_t i = 0; i < lf.n; ++i) lf.inv[lf.perm[i]] = i;
    lf.parent.resize(lf.n);
    lc.child_ptr.assign(lc.n + 1, 0);
    for (int64_t i = 0; i < lf.n; ++i) {
      lf.parent[i] = (int32_t)key[lf.perm[i]];
      lc.child_ptr[key[lf.perm[i]] + 1] += 1;
    }
    for (int64_t k = 0; k < lc.n; ++k) lc.child_ptr[k + 1] += lc.child_ptr[k];
  }
  // ---- level 0 operator in internal order: A0 = c M + A
  {
    HostLevel& l0 = h.lev[0];
    const int64_t ne = m.ne;
    l0.A.nrows = ne;
    l0.A.B = B;
    l0.A.rowptr.assign(ne + 1, 0);
    for (int64_t r = 0; r < ne; ++r) {
      int64_t e = l0.perm[r];
      l0.A.rowptr[r + 1] = l0.A.rowptr[r] + (m.A.rowptr[e + 1] - m.A.rowptr[e]);
    }
    l0.A.col.resize(l0.A.rowptr[ne]);
    l0.A.val.resize((size_t)l0.A.rowptr[ne] * B * B);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < ne; ++r) {
      const int64_t e = l0.perm[r];
      const int64_t s0 = m.A.rowptr[e], cnt = m.A.rowptr[e + 1] - s0;
      std::vector<std::pair<int64_t, int64_t>> cols(cnt);
      for (int64_t k = 0; k < cnt; ++k) cols[k] = {l0.inv[m.A.col[s0 + k]], s0 + k};
      std::sort(cols.begin(), cols.end());
      for (int64_t k = 0; k < cnt; ++k) {
        const int64_t dst = l0.A.rowptr[r] + k;
        l0.A.col[dst] = (int32_t)cols[k].first;
        double* out = &l0.A.val[(size_t)dst * B * B];
        std::memcpy(out, &m.A.val[(size_t)cols[k].second * B * B], sizeof(double) * B * B);
        if (cols[k].first == r)
          for (int i = 0; i < B * B; ++i) out[i] += c * m.Me[(size_t)e * B * B + i];
      }
    }
  }
  // ---- nodal points of level 0: physical GLL nodes of each element
  Tables1D t = make_tables(p, p + 2);
  const int n1 = p + 1, V = 1 << dim;
  {
    HostLevel& l0 = h.lev[0];
    l0.nodes.resize((size_t)l0.n * B * dim);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < l0.n; ++r) {
      const int64_t e = l0.perm[r];
      for (int i = 0; i < B; ++i) {
        double xi[3];
        int rr = i;
        for (int k = 0; k < dim; ++k) { xi[k] = t.gll[rr % n1]; rr /= n1; }
        for (int k = 0; k < dim; ++k) {
          double s = 0.0;
          for (int cc = 0; cc < V; ++cc) {
            double N = 1.0;
            for (int a = 0; a < dim; ++a) N *= ((cc >> a) & 1) ? xi[a] : 1.0 - xi[a];
            s += N * m.X[m.cells[e * V + cc] * dim + k];
          }
          l0.nodes[((size_t)r * B + i) * dim + k] = s;
        }
      }
    }
  }
  // ---- coarse levels
  for (int l = 0; l + 1 < L; ++l) {
    HostLevel& lf = h.lev[l];
    HostLevel& lc = h.lev[l + 1];
    // bounding boxes
    lc.lo.assign((size_t)lc.n * dim, 1e300);
    lc.hi.assign((size_t)lc.n * dim, -1e300);
    for (int64_t u = 0; u < lf.n; ++u) {
      const int64_t K = lf.parent[u];
      if (l == 0) {
        const int64_t e = lf.perm[u];
        for (int cc = 0; cc < V; ++cc)
          for (int k = 0; k < dim; ++k) {
            double x = m.X[m.cells[e * V + cc] * dim + k];
            lc.lo[K * dim + k] = std::min(lc.lo[K * dim + k], x);
            lc.hi[K * dim + k] = std::max(lc.hi[K * dim + k], x);
          }
      } else {
        for (int k = 0; k < dim; ++k) {
          lc.lo[K * dim + k] = std::min(lc.lo[K * dim + k], lf.lo[u * dim + k]);
          lc.hi[K * dim + k] = std::max(lc.hi[K * dim + k], lf.hi[u * dim + k]);
        }
      }
    }
    // prolongation blocks: P[u][i][j] = prod_k l_{j_k}((y_{u,i,k} - lo_k)/(hi_k - lo_k))
    lf.P.resize((size_t)lf.n * B * B);
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < lf.n; ++u) {
      const int64_t K = lf.parent[u];
      for (int i = 0; i < B; ++i) {
        double v[3][8], d[3][8];
        for (int k = 0; k < dim; ++k) {
          double eta = (lf.nodes[((size_t)u * B + i) * dim + k] - lc.lo[K * dim + k]) /
                       (lc.hi[K * dim + k] - lc.lo[K * dim + k]);
          lagrange_eval(t.gll.data(), n1, eta, v[k], d[k]);
        }
        for (int j = 0; j < B; ++j) {
          int rr = j;
          double val = 1.0;
          for (int k = 0; k < dim; ++k) { val *= v[k][rr % n1]; rr /= n1; }
          lf.P[((size_t)u * B + i) * B + j] = val;
        }
      }
    }
    if (o.direct) {
      int rc = direct_level_build(m, h, l + 1, c, lc.A, err);
      if (rc) return rc;
    } else {
      // Galerkin product, one coarse block row per thread
      std::vector<std::vector<int32_t>> rcols(lc.n);
      std::vector<std::vector<double>> rvals(lc.n);
#pragma omp parallel for schedule(dynamic, 4)
      for (int64_t K = 0; K < lc.n; ++K) {
        std::vector<int32_t> cols;
        std::vector<double> acc;
        std::vector<double> T((size_t)B * B);
        for (int64_t u = lc.child_ptr[K]; u < lc.child_ptr[K + 1]; ++u) {
          const double* Pu = &lf.P[(size_t)u * B * B];
          for (int64_t k = lf.A.rowptr[u]; k < lf.A.rowptr[u + 1]; ++k) {
            const int64_t v = lf.A.col[k];
            const int32_t Kp = lf.parent[v];
            size_t slot = 0;
            while (slot < cols.size() && cols[slot] != Kp) ++slot;
            if (slot == cols.size()) {
              cols.push_back(Kp);
              acc.resize(acc.size() + (size_t)B * B, 0.0);
            }
            gemm(&lf.A.val[(size_t)k * B * B], &lf.P[(size_t)v * B * B], T.data(), B);
            gemm_tn_acc(Pu, T.data(), &acc[slot * B * B], B);
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
      lc.A.nrows = lc.n;
      lc.A.B = B;
      lc.A.rowptr.assign(lc.n + 1, 0);
      for (int64_t K = 0; K < lc.n; ++K) lc.A.rowptr[K + 1] = lc.A.rowptr[K] + (int64_t)rcols[K].size();
      lc.A.col.resize(lc.A.rowptr[lc.n]);
      lc.A.val.resize((size_t)lc.A.rowptr[lc.n] * B * B);
      for (int64_t K = 0; K < lc.n; ++K) {
        std::copy(rcols[K].begin(), rcols[K].end(), lc.A.col.begin() + lc.A.rowptr[K]);
        std::copy(rvals[K].begin(), rvals[K].end(), lc.A.val.begin() + lc.A.rowptr[K] * B * B);
      }
    }
    // nodal points of level l+1: GLL nodes of the boxes
    lc.nodes.resize((size_t)lc.n * B * dim);
    for (int64_t K = 0; K < lc.n; ++K)
      for (int i = 0; i < B; ++i) {
        int rr = i;
        for (int k = 0; k < dim; ++k) {
          lc.nodes[((size_t)K * B + i) * dim + k] =
              lc.lo[K * dim + k] + t.gll[rr % n1] * (lc.hi[K * dim + k] - lc.lo[K * dim + k]);
          rr /= n1;
        }
      }
  }
  // ---- smoother blocks and Chebyshev bounds on every level but the coarsest
  for (int l = 0; l + 1 < L; ++l) {
    HostLevel& lv = h.lev[l];
    const int64_t n = lv.n;
    std::vector<double> Dblk((size_t)n * B * B, 0.0);
    lv.Dinv.assign((size_t)n * B * B, 0.0);
    int notspd = 0;
#pragma omp parallel for schedule(static) reduction(+ : notspd)
    for (int64_t u = 0; u < n; ++u) {
      const double* blk = nullptr;
      for (int64_t k = lv.A.rowptr[u]; k < lv.A.rowptr[u + 1]; ++k)
        if (lv.A.col[k] == u) blk = &lv.A.val[(size_t)k * B * B];
      if (!blk) { notspd += 1; continue; }
      double* Db = &Dblk[(size_t)u * B * B];
      double* Di = &lv.Dinv[(size_t)u * B * B];
      if (o.block_jacobi) {
        std::memcpy(Db, blk, sizeof(double) * B * B);
        std::vector<double> Lc(Db, Db + B * B), Li((size_t)B * B);
        if (!cholesky(Lc.data(), B)) { notspd += 1; continue; }
        lower_inverse(Lc.data(), Li.data(), B);
        // D^{-1} = L^{-T} L^{-1}
        for (int i = 0; i < B; ++i)
          for (int j = 0; j < B; ++j) {
            double s = 0.0;
            for (int k = std::max(i, j); k < B; ++k) s += Li[k * B + i] * Li[k * B + j];
            Di[i * B + j] = s;
          }
      } else {
        for (int i = 0; i < B; ++i) {
          Db[i * B + i] = blk[i * B + i];
          if (!(blk[i * B + i] > 0.0)) notspd += 1;
          Di[i * B + i] = 1.0 / blk[i * B + i];
        }
      }
    }
    if (notspd) { err = "a smoother block is not SPD on level " + std::to_string(l); return AGG_ENOTSPD; }
    // Lanczos on D^{-1} A in the D-inner product, v_i = sin(i+1) in the caller's numbering
    const int64_t N = n * B;
    const int msteps = (int)std::min<int64_t>(o.lanczos_steps, N);
    std::vector<double> v(N), vp(N, 0.0), w(N), Av(N), Dw(N);
    for (int64_t r = 0; r < n; ++r)
      for (int i = 0; i < B; ++i) v[r * B + i] = std::sin((double)(lv.perm[r] * B + i + 1));
    block_apply_host(Dblk, B, v.data(), Dw.data(), n);
    double nv = std::sqrt(dot(v, Dw));
    for (auto& x : v) x /= nv;
    std::vector<double> al, be;
    double beta = 0.0;
    for (int j = 0; j < msteps; ++j) {
      bsr_apply(lv.A, v.data(), Av.data());
      double alpha = dot(Av, v);
      block_apply_host(lv.Dinv, B, Av.data(), w.data(), n);
      for (int64_t i = 0; i < N; ++i) w[i] -= alpha * v[i] + beta * vp[i];
      al.push_back(alpha);
      if (j == msteps - 1) break;
      block_apply_host(Dblk, B, w.data(), Dw.data(), n);
      double b2 = dot(w, Dw);
      beta = std::sqrt(std::max(b2, 0.0));
      if (beta == 0.0) break;
      be.push_back(beta);
      vp = v;
      for (int64_t i = 0; i < N; ++i) v[i] = w[i] / beta;
    }
    be.resize(al.size() > 0 ? al.size() - 1 : 0);
    lv.lam_hat = tridiag_max_eig(al, be);
    lv.lam_max = o.safety * lv.lam_hat;
    lv.lam_min = lv.lam_max / o.range;
  }
  // ---- coarsest operator: dense Cholesky and the inverse factor
  {
    HostLevel& lc = h.lev[L - 1];
    const int64_t nc = lc.n * B;
    if (nc > 16384) { err = "coarsest level too large for the dense solve (> 16384 DoFs)"; return AGG_EINVAL; }
    h.nc = nc;
    std::vector<double> Ad((size_t)nc * nc, 0.0);
    for (int64_t r = 0; r < lc.n; ++r)
      for (int64_t k = lc.A.rowptr[r]; k < lc.A.rowptr[r + 1]; ++k) {
        const int64_t cc = lc.A.col[k];
        for (int i = 0; i < B; ++i)
          for (int j = 0; j < B; ++j)
            Ad[(r * B + i) * nc + cc * B + j] = lc.A.val[(size_t)k * B * B + i * B + j];
      }
    if (!cholesky(Ad.data(), nc)) { err = "coarsest operator is not SPD"; return AGG_ENOTSPD; }
    h.Linv.resize((size_t)nc * nc);
    lower_inverse(Ad.data(), h.Linv.data(), nc);
  }
  return AGG_OK;
}

}  // namespace aggmg
