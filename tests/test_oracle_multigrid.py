"""Pins of the oracle's agglomerated multigrid (Sections 5-6)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spl

from oracle import multigrid as mg
from oracle import refelem as re
from oracle import sipg
from paper_2602_16312_gb300 import workloads as W


def _disc(dim=2, n=8, p=2, jit=0.0, seed=6):
    mesh = W.box_mesh(dim, n, jitter=jit, seed=seed)
    if dim == 2:
        D = W.conductivity_from_fibres(W.planar_fibres(mesh.n_elements, 30.0), 1.2e-3, 2.5e-4)
    else:
        D = W.conductivity_from_fibres(W.rotating_fibres_z(mesh.centroids()), 1.2e-3, 2.5e-4)
    return mesh, sipg.assemble(mesh.vertices, mesh.elements, D, p, 1, 10.0)


def _q_tensor(y):          # in Q_2 (degree 2 per variable), not in P_2
    return y[..., 0] ** 2 * y[..., 1] - 0.5 * y[..., 1] ** 2 + y[..., 0] * y[..., 1] + 0.2


def _q_total(y):           # total degree <= 2
    return y[..., 0] ** 2 - 0.5 * y[..., 1] ** 2 + 0.7 * y[..., 0] * y[..., 1] - y[..., 1] + 0.2


@pytest.mark.parametrize("jit,q", [(0.0, _q_tensor), (0.2, _q_total)])
def test_prolongation_reproduces_polynomials(jit, q):
    mesh, disc = _disc(jit=jit)
    maps = W.block_hierarchy(mesh.grid_shape, (2, 2), 3)
    p = 2
    y0 = sipg.nodal_points(mesh.vertices, mesh.elements, p)
    lo1, hi1 = mg.level1_boxes(mesh.vertices, mesh.elements, maps[0].astype(np.int64))
    P1 = mg.prolongation(y0, maps[0].astype(np.int64), lo1, hi1, p)
    y1 = mg.box_nodal_points(lo1, hi1, p)
    np.testing.assert_allclose(P1 @ q(y1).ravel(), q(y0).ravel(), atol=1e-13)
    np.testing.assert_allclose(P1 @ np.ones(P1.shape[1]), 1.0, atol=1e-14)
    # levels >= 1 are exactly nested: Q_p reproduced even on jittered meshes
    lo2, hi2 = mg.coarser_boxes(lo1, hi1, maps[1].astype(np.int64))
    P2 = mg.prolongation(y1, maps[1].astype(np.int64), lo2, hi2, p)
    y2 = mg.box_nodal_points(lo2, hi2, p)
    np.testing.assert_allclose(P2 @ _q_tensor(y2).ravel(), _q_tensor(y1).ravel(), atol=1e-13)
    # every row of a block belongs to exactly one parent
    assert np.all(np.diff(P1.indptr) == 9)


@pytest.mark.parametrize("dim,jit", [(2, 0.2), (3, 0.15)])
def test_galerkin_coarse_operators(dim, jit):
    mesh, disc = _disc(dim=dim, n=4 if dim == 3 else 8, p=2 if dim == 2 else 1, jit=jit)
    maps = W.block_hierarchy(mesh.grid_shape, (2,) * dim, 3)
    h = mg.build_hierarchy(disc, 20.0, maps)
    Adiff = disc.A                                   # c = 0: diffusion part only
    for l, lev in enumerate(h.levels[1:]):
        A = lev.A.toarray()
        s = np.abs(A).max()
        assert np.abs(A - A.T).max() <= 1e-13 * s
        assert np.linalg.eigvalsh(A).min() > 0.0
        Adiff = mg.galerkin(Adiff, h.levels[l].P)
        Ad = Adiff.toarray()
        assert np.abs(Ad @ np.ones(Ad.shape[0])).max() <= 1e-12 * np.abs(Ad).max()
    for lev in h.levels[:-1]:
        eye = np.einsum("eij,ejk->eik", lev.Dinv, lev.Dblocks)
        np.testing.assert_allclose(eye, np.broadcast_to(np.eye(lev.B), eye.shape), atol=1e-12)


def test_chebyshev_error_propagator_is_scaled_T3():
    """Error propagator of the degree-3 Chebyshev iteration equals
    T_3((theta - lambda)/delta) / T_3(theta/delta) of D^{-1} A."""
    mesh, disc = _disc(n=3, p=1)
    A = disc.A0(20.0)
    Db = mg.diagonal_blocks(A, disc.B)
    Dinv = np.linalg.inv(Db)
    lmax = 1.2 * mg.lanczos_max_eig(A, Db)
    lmin = lmax / 20.0
    Ad = A.toarray()
    Dfull = sla.block_diag(*Db)
    lam, V = sla.eigh(Ad, Dfull)                    # D^{-1} A = V diag(lam) V^{-1}
    th, de = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    T3 = lambda x: 4 * x ** 3 - 3 * x
    pol = T3((th - lam) / de) / T3(th / de)
    E_expect = V @ np.diag(pol) @ np.linalg.inv(V)
    n = Ad.shape[0]
    E = np.stack([mg.chebyshev(A, Dinv, np.zeros(n), np.eye(n)[:, j], lmin, lmax) for j in range(n)], 1)
    np.testing.assert_allclose(E, E_expect, atol=1e-12)
    # started from zero with right-hand side b: x = (I - p(D^-1 A)) A^{-1} b
    b = np.random.default_rng(1).standard_normal(n)
    x = mg.chebyshev(A, Dinv, b, None, lmin, lmax, x_is_zero=True)
    np.testing.assert_allclose(x, (np.eye(n) - E_expect) @ np.linalg.solve(Ad, b), atol=1e-10)


def test_lanczos_exact_when_steps_cover_dimension():
    mesh, disc = _disc(n=1, p=1)                     # 4 DoFs
    A = disc.A0(20.0)
    Db = mg.diagonal_blocks(A, disc.B)
    lam = sla.eigh(A.toarray(), sla.block_diag(*Db), eigvals_only=True).max()
    assert abs(mg.lanczos_max_eig(A, Db, 12) - lam) <= 1e-12 * lam
    # and a lower bound that is tight after 12 steps on a larger problem
    mesh, disc = _disc(n=6, p=2)
    A = disc.A0(20.0)
    Db = mg.diagonal_blocks(A, disc.B)
    lam = sla.eigh(A.toarray(), sla.block_diag(*Db), eigvals_only=True).max()
    est = mg.lanczos_max_eig(A, Db, 12)
    assert est <= lam * (1 + 1e-12) and est >= 0.9 * lam


def _vcycle_matrix(h, n):
    return np.stack([mg.vcycle(h, np.eye(n)[:, j]) for j in range(n)], 1)


def test_vcycle_symmetric_positive_and_one_level_exact():
    mesh, disc = _disc(n=8, p=1, jit=0.2)
    maps = W.block_hierarchy(mesh.grid_shape, (2, 2), 3)
    h = mg.build_hierarchy(disc, 20.0, maps)
    n = disc.n
    Bm = _vcycle_matrix(h, n)
    assert np.abs(Bm - Bm.T).max() <= 1e-12 * np.abs(Bm).max()
    assert np.linalg.eigvalsh(0.5 * (Bm + Bm.T)).min() > 0.0
    h1 = mg.build_hierarchy(disc, 20.0, [])
    A = disc.A0(20.0).toarray()
    np.testing.assert_allclose(_vcycle_matrix(h1, n) @ A, np.eye(n), atol=1e-10)
    b = np.random.default_rng(2).standard_normal(n)
    res = mg.pcg(disc.A0(20.0), b, np.zeros(n), lambda r: mg.vcycle(h1, r), 1e-10)
    assert res.iterations == 1


def test_pcg_matches_direct_solve():
    mesh, disc = _disc(n=8, p=2, jit=0.2)
    maps = mg_maps = W.rcb_hierarchy(mesh, 4, 3)
    h = mg.build_hierarchy(disc, 20.0, mg_maps)
    A = disc.A0(20.0)
    b = np.random.default_rng(3).standard_normal(disc.n)
    x0 = np.random.default_rng(4).standard_normal(disc.n)
    res = mg.pcg(A, b, x0, lambda r: mg.vcycle(h, r), 1e-12)
    x = spl.spsolve(A.tocsc(), b)
    assert res.converged and res.iterations < 30
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)
