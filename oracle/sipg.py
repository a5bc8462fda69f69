"""SIPG-DG discretisation of the monodomain diffusion operator (Section 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Computes, in float64, for a conforming quad/hex mesh with multilinear
element maps and the DG space of tensor Q_p polynomials on GLL nodes:
  * the mass matrix M, (M)_ij = m_h(phi_j, phi_i) = int phi_i phi_j
    (Section 3, Eq. matrices);
  * the SIPG stiffness A, (A)_ij = a_h(phi_j, phi_i) (Section 3, the a_h form
    and the penalty sigma = alpha n^T D n):
      a_h(u, v) = sum_K int_K D grad u . grad v
                - sum_{F interior} int_F ( {D grad u}.[v] + {D grad v}.[u] )
                + sum_{F interior} int_F sigma [u].[v]
    with [v] = v+ n+ + v- n-, {q} = (q+ + q-)/2. Boundary faces contribute
    nothing (homogeneous Neumann, Section 2.2).
  * A0 = c M + A, the matrix of Eq. fully_discrete (c = 3 chi C_m / (2 dt) for
    BDF2, c = chi C_m / dt for the backward-Euler form used by the workloads).

Readings where the paper is silent or garbled:
  * The printed a_h puts the penalty inside the negated bracket, which would
    make A indefinite; the standard symmetric interior penalty sign (+sigma)
    is used. Pinned by the positive semi-definiteness test.
  * alpha = C_pen max(|F|/|K+|, |F|/|K-|), C_pen = p(p+1) (paper) or
    penalty_coeff * p^2 (penalty_mode 1); D in n^T D n is the face average
    (D+ + D-)/2, evaluated at every face quadrature point.
  * Quadrature: Gauss-Legendre with p + 1 + quad_extra points per direction
    (default p + 2) for volumes and faces.

Pins (tests/test_oracle_sipg.py): textbook 1D mass/stiffness Kronecker forms
on Cartesian meshes; 1^T M 1 = |Omega|; symmetry; A 1 = 0; A PSD on jittered
meshes; consistency a_h(q, v) = int_{dOmega} (D grad q . n) v for linear q;
h^{p+1} L2 convergence on a manufactured solution.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import refelem as re


@dataclass
class Discretisation:
    dim: int
    p: int
    B: int                       # DoFs per element, (p+1)^dim
    n_elements: int
    M: sp.csr_matrix
    A: sp.csr_matrix
    Me: np.ndarray               # (E, B, B) element mass blocks
    volumes: np.ndarray          # (E,)
    vertices: np.ndarray
    elements: np.ndarray

    @property
    def n(self) -> int:
        return self.n_elements * self.B

    def A0(self, mass_coeff: float) -> sp.csr_matrix:
        return (mass_coeff * self.M + self.A).tocsr()


def _geometry(X, N, dN):
    """Multilinear map x(xi) = sum_v X_v N_v(xi) and its Jacobian
    J[k, l] = dx_k / dxi_l at the points of N/dN. X (E, V, d)."""
    x = np.einsum("qv,evk->eqk", N, X)
    J = np.einsum("qvl,evk->eqkl", dN, X)
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0.0):
        raise ValueError("element with non-positive Jacobian")
    Jinv = np.linalg.inv(J)
    return x, J, detJ, Jinv


def _physical_gradients(Jinv, grad_hat):
    """grad phi_i = J^{-T} grad_hat phi_i: component k = sum_l Jinv[l, k] d_l phi_i.
    Jinv (E, Q, d, d), grad_hat (B, Q, d) -> (E, Q, B, d)."""
    return np.einsum("eqlk,iql->eqik", Jinv, grad_hat)


def volume_matrices(vertices, elements, D, p, quad_extra=1, chunk=32768):
    """Element mass and stiffness blocks (E, B, B) and element volumes:
      M_e[i,j] = sum_q w_q |J| phi_i phi_j
      K_e[i,j] = sum_q w_q |J| (J^{-T} grad phi_i)^T D_e (J^{-T} grad phi_j)."""
    dim = vertices.shape[1]
    q = p + 1 + quad_extra
    x1, w1 = re.gauss_rule(q)
    xi = re.tensor_points(x1, dim)
    w = re.tensor_weights(w1, dim)
    phi, grad_hat = re.tensor_basis(p, dim, xi)
    N, dN = re.multilinear_shape(dim, xi)
    E = elements.shape[0]
    B = phi.shape[0]
    Me = np.empty((E, B, B))
    Ke = np.empty((E, B, B))
    vol = np.empty(E)
    for s in range(0, E, chunk):
        X = vertices[elements[s:s + chunk]]
        _, _, detJ, Jinv = _geometry(X, N, dN)
        G = _physical_gradients(Jinv, grad_hat)
        wJ = w[None, :] * detJ
        Me[s:s + chunk] = np.einsum("eq,iq,jq->eij", wJ, phi, phi, optimize=True)
        # the same sum, contracted in two steps: (D grad phi_j) first, then
        # sum_q w |J| grad phi_i . (D grad phi_j)
        DG = np.einsum("ekm,eqjm->eqjk", D[s:s + chunk], G)
        Ke[s:s + chunk] = np.einsum("eq,eqik,eqjk->eij", wJ, G, DG, optimize=True)
        vol[s:s + chunk] = wJ.sum(axis=1)
    return Me, Ke, vol


def face_corner_list(dim, f):
    """Element corners on local face f = 2k + s (xi_k = s), ordered by the
    face-corner index over the remaining axes (lowest axis fastest)."""
    k, s = divmod(f, 2)
    others = [a for a in range(dim) if a != k]
    out = []
    for m in range(2 ** (dim - 1)):
        c = s << k
        for j, a in enumerate(others):
            c |= ((m >> j) & 1) << a
        out.append(c)
    return out


def face_embed(dim, f, t):
    """Reference points of face f = 2k + s from face coordinates t (Q, d-1)."""
    k, s = divmod(f, 2)
    others = [a for a in range(dim) if a != k]
    xi = np.empty((t.shape[0], dim))
    xi[:, k] = float(s)
    for j, a in enumerate(others):
        xi[:, a] = t[:, j]
    return xi


def find_faces(elements, dim):
    """Interior faces by matching the sorted vertex ids of local faces.

    Returns (ep, fp, em, fm, match): element/local face of the + side (the
    smaller element index) and of the - side, and match[F, m] = the element
    corner of e- that carries the vertex of face-corner m of e+."""
    E = elements.shape[0]
    nf = 2 * dim
    fc = [face_corner_list(dim, f) for f in range(nf)]
    ids = np.stack([elements[:, fc[f]] for f in range(nf)], axis=1)   # (E, nf, V_f)
    ids = ids.reshape(E * nf, -1)
    key = np.sort(ids, axis=1)
    order = np.lexsort(key.T[::-1])
    ks = key[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    a = order[:-1][same]
    b = order[1:][same]
    ea, fa = np.divmod(a, nf)
    eb, fb = np.divmod(b, nf)
    swap = ea > eb
    ep = np.where(swap, eb, ea)
    fp = np.where(swap, fb, fa)
    em = np.where(swap, ea, eb)
    fm = np.where(swap, fa, fb)
    ids_p = ids[ep * nf + fp]
    ids_m = ids[em * nf + fm]
    nvf = ids.shape[1]
    match = np.empty((len(ep), nvf), dtype=np.int64)
    fc_arr = np.array(fc)
    for m in range(nvf):
        pos = np.argmax(ids_m == ids_p[:, m:m + 1], axis=1)
        assert np.all(ids_m[np.arange(len(ep)), pos] == ids_p[:, m])
        match[:, m] = fc_arr[fm, pos]
    return ep, fp, em, fm, match


def face_matrices(vertices, elements, D, p, volumes, c_pen, quad_extra=1, chunk=65536, side=None):
    """Face blocks of the SIPG form on every interior face.

    Returns (ep, em, blocks) with blocks (F, 2, 2, B, B): blocks[F, si, sj] is
    the contribution to rows of side si and columns of side sj (0 = +, 1 = -):
      sum_q w_q dS_q [ -1/2 sgn_i phi_i (D_sj grad phi_j . n)
                       -1/2 sgn_j phi_j (D_si grad phi_i . n)
                       + sigma_q sgn_i sgn_j phi_i phi_j ]
    with n the unit outward normal of the + element, sgn(+) = 1, sgn(-) = -1,
    sigma_q = c_pen max(|F|/|K+|, |F|/|K-|) n^T ((D+ + D-)/2) n.

    side = 0 (1) keeps only the terms built with D+ (D-): the blocks are linear
    in (D+, D-) jointly, so the two parts add up to the full face blocks."""
    dim = vertices.shape[1]
    q = p + 1 + quad_extra
    x1, w1 = re.gauss_rule(q)
    t = re.tensor_points(x1, dim - 1) if dim > 1 else np.zeros((1, 0))
    wt = re.tensor_weights(w1, dim - 1)
    Nf, _ = re.multilinear_shape(dim - 1, t)                        # (Q, Vf)
    ep, fp, em, fm, match = find_faces(elements, dim)
    F = len(ep)
    Q = t.shape[0]
    B = (p + 1) ** dim
    corner_xi = np.array([[(c >> k) & 1 for k in range(dim)] for c in range(2 ** dim)], float)
    blocks = np.empty((F, 2, 2, B, B))
    for s in range(0, F, chunk):
        sl = slice(s, s + chunk)
        nF = len(ep[sl])
        xi_p = np.stack([face_embed(dim, f, t) for f in range(2 * dim)])[fp[sl]]   # (nF, Q, d)
        xi_m = np.einsum("qm,fmk->fqk", Nf, corner_xi[match[sl]])
        pts_p = xi_p.reshape(-1, dim)
        pts_m = xi_m.reshape(-1, dim)
        Np, dNp = re.multilinear_shape(dim, pts_p)
        Nm, dNm = re.multilinear_shape(dim, pts_m)
        Xp = vertices[elements[ep[sl]]]
        Xm = vertices[elements[em[sl]]]
        xp = np.einsum("fqv,fvk->fqk", Np.reshape(nF, Q, -1), Xp)
        xm = np.einsum("fqv,fvk->fqk", Nm.reshape(nF, Q, -1), Xm)
        if np.max(np.abs(xp - xm)) > 1e-12 * max(1.0, np.max(np.abs(xp))):
            raise ValueError("face quadrature points do not coincide")
        Jp = np.einsum("fqvl,fvk->fqkl", dNp.reshape(nF, Q, -1, dim), Xp)
        Jm = np.einsum("fqvl,fvk->fqkl", dNm.reshape(nF, Q, -1, dim), Xm)
        detp = np.linalg.det(Jp)
        Jinvp = np.linalg.inv(Jp)
        Jinvm = np.linalg.inv(Jm)
        kf, sf = np.divmod(fp[sl], 2)
        nhat = np.zeros((nF, dim))
        nhat[np.arange(nF), kf] = 2.0 * sf - 1.0
        # J^{-T} nhat: component k = sum_l Jinv[l, k] nhat_l
        nvec = np.einsum("fqlk,fl->fqk", Jinvp, nhat)
        nlen = np.linalg.norm(nvec, axis=2)
        n = nvec / nlen[..., None]
        wdS = wt[None, :] * detp * nlen                                   # (nF, Q)
        area = wdS.sum(axis=1)
        alpha = c_pen * np.maximum(area / volumes[ep[sl]], area / volumes[em[sl]])
        Dp = D[ep[sl]]
        Dm = D[em[sl]]
        if side == 0:
            Dm = np.zeros_like(Dm)
        elif side == 1:
            Dp = np.zeros_like(Dp)
        Dbar = 0.5 * (Dp + Dm)
        sigma = alpha[:, None] * np.einsum("fqk,fkm,fqm->fq", n, Dbar, n)
        phi_p, gh_p = re.tensor_basis(p, dim, pts_p)
        phi_m, gh_m = re.tensor_basis(p, dim, pts_m)
        phi_p = phi_p.reshape(B, nF, Q).transpose(1, 2, 0)                # (nF, Q, B)
        phi_m = phi_m.reshape(B, nF, Q).transpose(1, 2, 0)
        gh_p = gh_p.reshape(B, nF, Q, dim).transpose(1, 2, 0, 3)          # (nF, Q, B, d)
        gh_m = gh_m.reshape(B, nF, Q, dim).transpose(1, 2, 0, 3)
        g_p = np.einsum("fqlk,fqil->fqik", Jinvp, gh_p)
        g_m = np.einsum("fqlk,fqil->fqik", Jinvm, gh_m)
        flux_p = np.einsum("fqik,fkm,fqm->fqi", g_p, Dp, n)               # D+ grad phi . n
        flux_m = np.einsum("fqik,fkm,fqm->fqi", g_m, Dm, n)
        phis = (phi_p, phi_m)
        fluxes = (flux_p, flux_m)
        sgn = (1.0, -1.0)
        for si in range(2):
            for sj in range(2):
                blk = (-0.5 * sgn[si] * np.einsum("fq,fqi,fqj->fij", wdS, phis[si], fluxes[sj], optimize=True)
                       - 0.5 * sgn[sj] * np.einsum("fq,fqj,fqi->fij", wdS, phis[sj], fluxes[si], optimize=True)
                       + sgn[si] * sgn[sj] * np.einsum("fq,fqi,fqj->fij", wdS * sigma,
                                                       phis[si], phis[sj], optimize=True))
                blocks[sl, si, sj] = blk
    return ep, em, blocks


def penalty_constant(p, penalty_mode, penalty_coeff):
    """C_pen: p(p+1) (the paper's alpha) or penalty_coeff * p^2."""
    return float(p * (p + 1)) if penalty_mode == 0 else float(penalty_coeff) * p * p


def _block_csr(E, B, diag, rows, cols, offd):
    """Global matrix from element diagonal blocks (E, B, B) and off-diagonal
    blocks offd[k] at block position (rows[k], cols[k])."""
    ii, jj = np.meshgrid(np.arange(B), np.arange(B), indexing="ij")
    r_d = (np.arange(E)[:, None, None] * B + ii).ravel()
    c_d = (np.arange(E)[:, None, None] * B + jj).ravel()
    r_o = (rows[:, None, None] * B + ii).ravel()
    c_o = (cols[:, None, None] * B + jj).ravel()
    r = np.concatenate([r_d, r_o])
    c = np.concatenate([c_d, c_o])
    v = np.concatenate([diag.ravel(), offd.ravel()])
    return sp.csr_matrix((v, (r, c)), shape=(E * B, E * B))


def assemble(vertices, elements, D, p, penalty_mode=0, penalty_coeff=10.0, quad_extra=1):
    """Mass M and SIPG stiffness A of the mesh (Section 3)."""
    vertices = np.asarray(vertices, dtype=np.float64)
    elements = np.asarray(elements, dtype=np.int64)
    D = np.asarray(D, dtype=np.float64)
    dim = vertices.shape[1]
    E = elements.shape[0]
    B = (p + 1) ** dim
    Me, Ke, vol = volume_matrices(vertices, elements, D, p, quad_extra)
    c_pen = penalty_constant(p, penalty_mode, penalty_coeff)
    ep, em, fb = face_matrices(vertices, elements, D, p, vol, c_pen, quad_extra)
    diag = Ke.copy()
    np.add.at(diag, ep, fb[:, 0, 0])
    np.add.at(diag, em, fb[:, 1, 1])
    rows = np.concatenate([ep, em])
    cols = np.concatenate([em, ep])
    offd = np.concatenate([fb[:, 0, 1], fb[:, 1, 0]])
    A = _block_csr(E, B, diag, rows, cols, offd)
    M = _block_csr(E, B, Me, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((0, B, B)))
    return Discretisation(dim, p, B, E, M, A, Me, vol, vertices, elements)


def nodal_points(vertices, elements, p):
    """Physical GLL nodes of every element, (E, B, d): x_e(xi_i)."""
    dim = vertices.shape[1]
    xi = re.tensor_points(re.gll_nodes(p), dim)
    N, _ = re.multilinear_shape(dim, xi)
    return np.einsum("iv,evk->eik", N, vertices[elements])


def attributed_forms(vertices, elements, D, p, penalty_mode=0, penalty_coeff=10.0, quad_extra=1):
    """Split of the SIPG stiffness into per-element parts, A = sum_e A_e:
    A_e is the volume form of e plus, on each interior face of e, the face
    terms built with D_e (consistency terms of e's side, half the penalty).
    Returns (Ke, ep, em, Yp, Ym) with Yp/Ym (F, 2, 2, B, B) the face blocks
    attributed to the + and - element. A_e is the derivative of A with respect
    to a scale factor s_e of D_e, at s_e = 1 (A is linear in each D_e)."""
    vertices = np.asarray(vertices, dtype=np.float64)
    elements = np.asarray(elements, dtype=np.int64)
    D = np.asarray(D, dtype=np.float64)
    Me, Ke, vol = volume_matrices(vertices, elements, D, p, quad_extra)
    c_pen = penalty_constant(p, penalty_mode, penalty_coeff)
    ep, em, Yp = face_matrices(vertices, elements, D, p, vol, c_pen, quad_extra, side=0)
    _, _, Ym = face_matrices(vertices, elements, D, p, vol, c_pen, quad_extra, side=1)
    return Ke, ep, em, Yp, Ym


def attributed_bilinear(forms, lam, u, B):
    """g_e = lam^T A_e u for every element (forms from attributed_forms)."""
    Ke, ep, em, Yp, Ym = forms
    E = Ke.shape[0]
    L = lam.reshape(E, B)
    U = u.reshape(E, B)
    g = np.einsum("ei,eij,ej->e", L, Ke, U)
    for Y, owner in ((Yp, ep), (Ym, em)):
        val = (np.einsum("fi,fij,fj->f", L[ep], Y[:, 0, 0], U[ep])
               + np.einsum("fi,fij,fj->f", L[ep], Y[:, 0, 1], U[em])
               + np.einsum("fi,fij,fj->f", L[em], Y[:, 1, 0], U[ep])
               + np.einsum("fi,fij,fj->f", L[em], Y[:, 1, 1], U[em]))
        np.add.at(g, owner, val)
    return g


def locate_points(vertices, elements, p, points, tol=1e-12):
    """Element and reference coordinates of each point (Newton on the
    multilinear map, among elements whose vertex box contains the point), and
    the interpolation weights phi_i(xi) of its element: returns (elem, W) with
    u_h(point) = sum_i W[s, i] u[elem[s]*B + i]."""
    dim = vertices.shape[1]
    X = vertices[elements]
    lo, hi = X.min(axis=1), X.max(axis=1)
    elem = np.empty(len(points), dtype=np.int64)
    xis = np.empty((len(points), dim))
    for s, x in enumerate(points):
        cand = np.nonzero(np.all((lo - 1e-12 <= x) & (x <= hi + 1e-12), axis=1))[0]
        found = False
        for e in cand:
            xi = np.full(dim, 0.5)
            for _ in range(50):
                N, dN = re.multilinear_shape(dim, xi[None])
                r = N[0] @ X[e] - x
                J = np.einsum("vl,vk->kl", dN[0], X[e])
                step = np.linalg.solve(J, r)
                xi = xi - step
                if np.max(np.abs(step)) < 1e-15:
                    break
            if np.all(xi >= -1e-10) and np.all(xi <= 1 + 1e-10):
                elem[s] = e
                xis[s] = np.clip(xi, 0.0, 1.0)
                found = True
                break
        if not found:
            raise ValueError(f"point {s} is outside the mesh")
    phi, _ = re.tensor_basis(p, dim, xis)
    return elem, phi.T
