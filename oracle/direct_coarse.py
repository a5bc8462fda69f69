"""Non-inherited coarse operators (Section 5.1): the SIPG bilinear form
assembled directly on an agglomerated level.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 5.1 names two ways to obtain the coarse operators: the inherited one
(Galerkin products, Eq. inherited_matrices; oracle.multigrid) and the
non-inherited one, where the bilinear forms are assembled on every
agglomerated level by numerical integration over the agglomerates, using the
original mesh for the quadrature. This module writes the latter out:

  A_l[(K,i),(K',j)] = sum over fine elements e in K (K = K'):
        int_e (grad phi_i^K)^T D_e grad phi_j^K + c phi_i^K phi_j^K
    + sum over fine interior faces F between elements of different
      agglomerates (K = agglomerate of e+, K' of e-), the SIPG face terms of
      oracle.sipg.face_matrices with the coarse functions:
        -1/2 sgn_i phi_i (D_sj grad phi_j . n) - 1/2 sgn_j phi_j (D_si grad phi_i . n)
        + sigma sgn_i sgn_j phi_i phi_j,
  phi^K the Q_p Lagrange (GLL) basis of the agglomerate's bounding box
  (the coarse space of Section 5.1), evaluated at the fine quadrature points.

Readings (the paper does not write the non-inherited form out):
  * Gauss-Legendre quadrature of the fine elements and faces, p + 1 +
    quad_extra points per direction, as on level 0.
  * Penalty on the polytopic face F_KK' (all fine faces between K and K'):
    sigma = C_pen max(|F_KK'|/|K|, |F_KK'|/|K'|) n^T ((D+ + D-)/2) n per fine
    face point, with |K| the agglomerate's measure: the paper's
    alpha = p(p+1)|F|/|K| on the polytopic level, i.e. scaled by the coarse
    size instead of the fine one that the inherited operator carries.
    With one element per agglomerate it reduces to the level-0 penalty.
  * Boundary faces contribute nothing (homogeneous Neumann).
"""
import numpy as np
import scipy.sparse as sp

from . import refelem as re
from . import sipg


def box_basis_grad(lo, hi, p, y):
    """Values (n, m, B) and physical gradients (n, m, B, d) of the Q_p box
    basis of boxes (lo, hi) (n, d) at points y (n, m, d)."""
    n, m, dim = y.shape
    nodes = re.gll_nodes(p)
    idx = re.multi_indices(dim, p + 1)
    L = hi - lo
    eta = (y - lo[:, None, :]) / L[:, None, :]
    vals, ders = [], []
    for k in range(dim):
        v, d = re.lagrange_1d(nodes, eta[:, :, k].ravel())
        vals.append(v.reshape(p + 1, n, m).transpose(1, 2, 0))                   # (n, m, p+1)
        ders.append(d.reshape(p + 1, n, m).transpose(1, 2, 0) / L[:, None, k:k + 1])
    B = idx.shape[0]
    phi = np.ones((n, m, B))
    for k in range(dim):
        phi *= vals[k][:, :, idx[:, k]]
    grad = np.ones((n, m, B, dim))
    for k in range(dim):
        for kk in range(dim):
            grad[:, :, :, k] *= (ders[kk] if kk == k else vals[kk])[:, :, idx[:, kk]]
    return phi, grad


def level_operator(vertices, elements, D, p, mass_coeff, c_pen, unit, lo, hi, quad_extra=1):
    """The level's operator c M_l + A_l assembled on the agglomerates:
    unit[e] = agglomerate (in [0, len(lo))) of fine element e; lo, hi = the
    agglomerates' bounding boxes. Returns a CSR matrix (n_l B) x (n_l B)."""
    vertices = np.asarray(vertices, dtype=np.float64)
    elements = np.asarray(elements, dtype=np.int64)
    unit = np.asarray(unit, dtype=np.int64)
    dim = vertices.shape[1]
    B = (p + 1) ** dim
    nK = lo.shape[0]
    q = p + 1 + quad_extra
    x1, w1 = re.gauss_rule(q)
    # ---- volume terms over every fine element of each agglomerate
    xi = re.tensor_points(x1, dim)
    w = re.tensor_weights(w1, dim)
    N, dN = re.multilinear_shape(dim, xi)
    x, _, detJ, _ = sipg._geometry(vertices[elements], N, dN)
    wJ = w[None, :] * detJ
    phi, g = box_basis_grad(lo[unit], hi[unit], p, x)
    Dg = np.einsum("ekm,eqjm->eqjk", D, g)
    vol_e = (np.einsum("eq,eqik,eqjk->eij", wJ, g, Dg, optimize=True)
             + mass_coeff * np.einsum("eq,eqi,eqj->eij", wJ, phi, phi, optimize=True))
    diag = np.zeros((nK, B, B))
    np.add.at(diag, unit, vol_e)
    volK = np.zeros(nK)
    np.add.at(volK, unit, wJ.sum(axis=1))
    # ---- face terms on the fine faces between different agglomerates
    ep, fp, em, fm, match = sipg.find_faces(elements, dim)
    sel = unit[ep] != unit[em]
    ep, fp, em, match = ep[sel], fp[sel], em[sel], match[sel]
    rows, cols, offd = [], [], []
    if len(ep):
        t = re.tensor_points(x1, dim - 1) if dim > 1 else np.zeros((1, 0))
        wt = re.tensor_weights(w1, dim - 1)
        Nf, _ = re.multilinear_shape(dim - 1, t)
        F, Q = len(ep), t.shape[0]
        corner_xi = np.array([[(c >> k) & 1 for k in range(dim)] for c in range(2 ** dim)], float)
        xi_p = np.stack([sipg.face_embed(dim, f, t) for f in range(2 * dim)])[fp]        # (F, Q, d)
        xi_m = np.einsum("qm,fmk->fqk", Nf, corner_xi[match])
        Np, dNp = re.multilinear_shape(dim, xi_p.reshape(-1, dim))
        Nm, _ = re.multilinear_shape(dim, xi_m.reshape(-1, dim))
        Xp, Xm = vertices[elements[ep]], vertices[elements[em]]
        xp = np.einsum("fqv,fvk->fqk", Np.reshape(F, Q, -1), Xp)
        xm = np.einsum("fqv,fvk->fqk", Nm.reshape(F, Q, -1), Xm)
        if np.max(np.abs(xp - xm)) > 1e-12 * max(1.0, np.max(np.abs(xp))):
            raise ValueError("face quadrature points do not coincide")
        Jp = np.einsum("fqvl,fvk->fqkl", dNp.reshape(F, Q, -1, dim), Xp)
        detp = np.linalg.det(Jp)
        Jinvp = np.linalg.inv(Jp)
        kf, sf = np.divmod(fp, 2)
        nhat = np.zeros((F, dim))
        nhat[np.arange(F), kf] = 2.0 * sf - 1.0
        nvec = np.einsum("fqlk,fl->fqk", Jinvp, nhat)
        nlen = np.linalg.norm(nvec, axis=2)
        n = nvec / nlen[..., None]
        wdS = wt[None, :] * detp * nlen
        # measure of each polytopic face F_KK' (all fine faces between K and K')
        Kp, Km = unit[ep], unit[em]
        lo_k, hi_k = np.minimum(Kp, Km), np.maximum(Kp, Km)
        pair, inv = np.unique(lo_k * nK + hi_k, return_inverse=True)
        areaKK = np.zeros(len(pair))
        np.add.at(areaKK, inv, wdS.sum(axis=1))
        area = areaKK[inv]
        alpha = c_pen * np.maximum(area / volK[Kp], area / volK[Km])
        Dp, Dm = D[ep], D[em]
        sigma = alpha[:, None] * np.einsum("fqk,fkm,fqm->fq", n, 0.5 * (Dp + Dm), n)
        phi_p, g_p = box_basis_grad(lo[Kp], hi[Kp], p, xp)
        phi_m, g_m = box_basis_grad(lo[Km], hi[Km], p, xp)
        flux_p = np.einsum("fqik,fkm,fqm->fqi", g_p, Dp, n)
        flux_m = np.einsum("fqik,fkm,fqm->fqi", g_m, Dm, n)
        phis, fluxes, sgn, units = (phi_p, phi_m), (flux_p, flux_m), (1.0, -1.0), (Kp, Km)
        for si in range(2):
            for sj in range(2):
                blk = (-0.5 * sgn[si] * np.einsum("fq,fqi,fqj->fij", wdS, phis[si], fluxes[sj], optimize=True)
                       - 0.5 * sgn[sj] * np.einsum("fq,fqj,fqi->fij", wdS, phis[sj], fluxes[si], optimize=True)
                       + sgn[si] * sgn[sj] * np.einsum("fq,fqi,fqj->fij", wdS * sigma, phis[si], phis[sj],
                                                       optimize=True))
                if si == sj:
                    np.add.at(diag, units[si], blk)
                else:
                    rows.append(units[si])
                    cols.append(units[sj])
                    offd.append(blk)
    # ---- block CSR (off-diagonal blocks of the same pair summed by the sparse constructor)
    ii, jj = np.meshgrid(np.arange(B), np.arange(B), indexing="ij")
    r_all = [(np.arange(nK)[:, None, None] * B + ii).ravel()]
    c_all = [(np.arange(nK)[:, None, None] * B + jj).ravel()]
    v_all = [diag.ravel()]
    for r, c, v in zip(rows, cols, offd):
        r_all.append((r[:, None, None] * B + ii).ravel())
        c_all.append((c[:, None, None] * B + jj).ravel())
        v_all.append(v.ravel())
    A = sp.coo_matrix((np.concatenate(v_all), (np.concatenate(r_all), np.concatenate(c_all))),
                      shape=(nK * B, nK * B))
    return A.tocsr()
