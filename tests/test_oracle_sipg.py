"""Pins of the oracle's SIPG discretisation (Section 3) against closed forms,
exact invariants and a manufactured solution."""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import refelem as re
from oracle import sipg
from paper_2602_16312_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_1d_lagrange.json")))


def textbook(p, h):
    g = GOLD[f"p{p}"]
    M = h * np.array(g["mass_num"], float) / g["mass_den"]
    K = np.array(g["stiff_num"], float) / (g["stiff_den"] * h)
    w = h * np.array(g["w_num"], float) / g["w_den"]
    return M, K, w


def kron_all(mats):
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(out, m)
    return out


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_cartesian_element_matrices_are_kronecker_products(dim, p):
    n = 3
    h = 1.0 / n
    mesh = W.box_mesh(dim, n)
    dvals = np.array([1.0, 0.37, 2.1])[:dim]
    D = np.broadcast_to(np.diag(dvals), (mesh.n_elements, dim, dim)).copy()
    Me, Ke, vol = sipg.volume_matrices(mesh.vertices, mesh.elements, D, p)
    M1, K1, _ = textbook(p, h)
    # flat index i = i0 + (p+1) i1 + ...: the x factor is the LAST Kronecker factor
    Mexp = kron_all([M1] * dim)
    Kexp = np.zeros_like(Mexp)
    for k in range(dim):
        facs = [M1] * dim
        facs[dim - 1 - k] = K1
        Kexp += dvals[k] * kron_all(facs)
    for e in (0, mesh.n_elements // 2, mesh.n_elements - 1):
        np.testing.assert_allclose(Me[e], Mexp, atol=1e-15)
        np.testing.assert_allclose(Ke[e], Kexp, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(vol, h ** dim, rtol=1e-13)


@pytest.mark.parametrize("dim,n,p,jit", [(2, 6, 2, 0.2), (3, 3, 2, 0.15), (2, 5, 3, 0.2)])
def test_mass_total_symmetry_and_constants(dim, n, p, jit):
    mesh = W.box_mesh(dim, n, jitter=jit, seed=4)
    if dim == 2:
        D = W.conductivity_from_fibres(W.planar_fibres(mesh.n_elements, 30.0), 1.2e-3, 2.5e-4)
    else:
        D = W.conductivity_from_fibres(W.rotating_fibres_z(mesh.centroids()), 1.2e-3, 2.5e-4)
    disc = sipg.assemble(mesh.vertices, mesh.elements, D, p, 1, 10.0)
    one = np.ones(disc.n)
    # 1^T M 1 = |Omega| = 1 (boundary vertices fixed)
    assert abs(one @ (disc.M @ one) - 1.0) < 1e-13
    A = disc.A.toarray()
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-14 * scale
    # pure Neumann: constants are in the kernel of the diffusion operator
    assert np.abs(A @ one).max() <= 1e-13 * scale
    # positive semi-definite with the 10 p^2 penalty
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= -1e-12 * scale
    assert np.sum(ev < 1e-12 * scale) == 1          # kernel is exactly the constants


def test_paper_penalty_indefinite_on_jittered_anisotropic_mesh():
    """Documents the reading: with C_pen = p(p+1) (the paper's alpha) the
    64x64 jittered mesh with 30-degree fibres has an element whose diagonal
    block of A0 = 20 M + A is indefinite, so A0 is not SPD; 10 p^2 fixes it.
    (A principal submatrix of an SPD matrix is SPD.)"""
    from oracle.multigrid import diagonal_blocks
    mesh = W.box_mesh(2, 64, jitter=0.2, seed=1)
    D = W.conductivity_from_fibres(W.planar_fibres(mesh.n_elements, 30.0), 1.2e-3, 2.5e-4)
    for mode, coeff, bad in ((0, 0.0, True), (1, 10.0, False)):
        disc = sipg.assemble(mesh.vertices, mesh.elements, D, 2, mode, coeff)
        lam = np.linalg.eigvalsh(diagonal_blocks(disc.A0(20.0), disc.B)).min()
        assert (lam < 0.0) == bad


def _boundary_flux_vector(dim, n, p, Fmap, Dc, g):
    """int_{dOmega} (D g . n) phi_i ds for the affine image x = F y of the unit
    grid, built from the logical grid and the textbook face weights."""
    h = 1.0 / n
    _, _, w1 = textbook(p, 1.0)                       # weights on the unit interval
    B = (p + 1) ** dim
    detF = np.linalg.det(Fmap)
    FinvT = np.linalg.inv(Fmap).T
    idx = re.multi_indices(dim, p + 1)
    eidx = re.multi_indices(dim, n)                   # element grid index, x fastest
    out = np.zeros(n ** dim * B)
    for e in range(n ** dim):
        for k in range(dim):
            for s in (0, 1):
                if eidx[e, k] != (0 if s == 0 else n - 1):
                    continue
                nvec = (2 * s - 1) * FinvT[:, k]
                flux = (Dc @ g) @ nvec * abs(detF) * h ** (dim - 1)
                for i in range(B):
                    if idx[i, k] != s * p:
                        continue
                    wt = np.prod([w1[idx[i, a]] for a in range(dim) if a != k])
                    out[e * B + i] += flux * wt
    return out


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_consistency_for_linear_functions(dim, p):
    """For linear q and constant D, a_h(q, v) = int_{dOmega} (D grad q . n) v:
    pins the signs of the consistency terms and the face normals."""
    n = 3
    mesh = W.box_mesh(dim, n)
    Fmap = np.eye(dim) + 0.25 * np.tri(dim, dim, -1) + 0.1 * np.tri(dim, dim, -1).T
    verts = mesh.vertices @ Fmap.T
    Dc = np.array([[1.3, 0.4, 0.1], [0.4, 0.7, -0.2], [0.1, -0.2, 0.9]])[:dim, :dim]
    D = np.broadcast_to(Dc, (mesh.n_elements, dim, dim)).copy()
    disc = sipg.assemble(verts, mesh.elements, D, p, 1, 10.0)
    g = np.array([0.7, -1.1, 0.4])[:dim]
    xn = sipg.nodal_points(verts, mesh.elements, p).reshape(-1, dim)
    q = xn @ g + 0.3
    expect = _boundary_flux_vector(dim, n, p, Fmap, Dc, g)
    np.testing.assert_allclose(disc.A @ q, expect, atol=1e-13)


def _load_and_error(verts, elems, p, f, u_exact, uh=None):
    dim = verts.shape[1]
    x1, w1 = re.gauss_rule(p + 3)
    xi = re.tensor_points(x1, dim)
    wq = re.tensor_weights(w1, dim)
    phi, _ = re.tensor_basis(p, dim, xi)
    N, dN = re.multilinear_shape(dim, xi)
    X = verts[elems]
    x = np.einsum("qv,evk->eqk", N, X)
    detJ = np.linalg.det(np.einsum("qvl,evk->eqkl", dN, X))
    wJ = wq * detJ
    if uh is None:
        return np.einsum("eq,iq,eq->ei", wJ, phi, f(x)).ravel()
    B = phi.shape[0]
    val = np.einsum("ei,iq->eq", uh.reshape(-1, B), phi)
    return np.sqrt(np.sum(wJ * (val - u_exact(x)) ** 2))


@pytest.mark.parametrize("p,jit", [(1, 0.0), (2, 0.0), (2, 0.2), (3, 0.1)])
def test_manufactured_solution_converges_at_order_p_plus_1(p, jit):
    dim = 2
    c = 1.0
    Dd = np.diag([1.0, 0.5])
    u_ex = lambda x: np.cos(np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1])
    f = lambda x: (c + np.pi ** 2 * (Dd[0, 0] + Dd[1, 1])) * u_ex(x)
    errs = []
    for n in (4, 8, 16):
        mesh = W.box_mesh(dim, n, jitter=jit, seed=5)
        D = np.broadcast_to(Dd, (mesh.n_elements, 2, 2)).copy()
        disc = sipg.assemble(mesh.vertices, mesh.elements, D, p, 1, 10.0)
        b = _load_and_error(mesh.vertices, mesh.elements, p, f, u_ex)
        uh = spl.spsolve(disc.A0(c).tocsc(), b)
        errs.append(_load_and_error(mesh.vertices, mesh.elements, p, f, u_ex, uh))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] >= p + 1 - 0.2, (errs, rates)


def test_face_matching_on_periodic_shell():
    # periodic seam: every element has 6 faces; interior + boundary counts add up
    wl = W.ventricle_shell(16, 8, 2, n_levels=2)
    ep, fp, em, fm, match = sipg.find_faces(wl.mesh.elements, 3)
    nu, nv, ns = wl.mesh.grid_shape
    interior = nu * (nv * ns) + nu * (nv - 1) * ns + nu * nv * (ns - 1)
    assert len(ep) == interior
