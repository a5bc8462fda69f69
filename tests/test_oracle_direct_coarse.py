"""Pins of the oracle's non-inherited coarse operators (oracle/direct_coarse.py,
Section 5.1): the SIPG form assembled on the agglomerates.

  * One element per agglomerate on an axis-aligned mesh: the box basis is
    the element's own basis and the polytopic penalty is the element's, so
    the operator is the level-0 operator c M + A of the fine assembly
    (an independent code path: oracle.sipg's element and face matrices).
  * Nested agglomerates of an axis-aligned mesh: the coarse space lies in
    the fine one and its functions have no jumps inside an agglomerate, so
    without penalty the direct operator equals the Galerkin product
    P^T A_0 P (oracle.multigrid's inherited operator).
  * Jittered anisotropic mesh, real agglomerates: symmetric, constants in
    the kernel of the diffusion part, positive semidefinite.
"""
import numpy as np
import pytest

from oracle import direct_coarse as dc
from oracle import multigrid as mg
from oracle import sipg
from paper_2602_16312_gb300 import workloads as W


def _mesh(dim, n, jitter=0.0, seed=None):
    mesh = W.box_mesh(dim, n, jitter=jitter, seed=seed)
    if dim == 2:
        D = W.conductivity_from_fibres(W.planar_fibres(mesh.n_elements, 30.0), 1.2e-3, 2.5e-4)
    else:
        D = W.conductivity_from_fibres(W.rotating_fibres_z(mesh.centroids()), 1.2e-3, 2.5e-4)
    return mesh, D


@pytest.mark.parametrize("dim,n,p", [(2, 4, 1), (2, 4, 2), (2, 3, 3), (3, 3, 1), (3, 3, 2)])
def test_one_element_per_agglomerate_gives_the_fine_operator(dim, n, p):
    mesh, D = _mesh(dim, n)
    c_pen = 4.0 * p * p
    disc = sipg.assemble(mesh.vertices, mesh.elements, D, p, 1, 4.0)
    X = mesh.vertices[mesh.elements]
    A = dc.level_operator(mesh.vertices, mesh.elements, D, p, 20.0, c_pen, np.arange(mesh.n_elements),
                          X.min(axis=1), X.max(axis=1))
    ref = disc.A0(20.0)
    assert abs(A - ref).max() <= 1e-13 * abs(ref).max()


@pytest.mark.parametrize("dim,n,f,p", [(2, 8, 2, 2), (2, 8, 4, 1), (3, 4, 2, 2)])
def test_nested_agglomerates_without_penalty_give_the_galerkin_product(dim, n, f, p):
    mesh, D = _mesh(dim, n)
    maps = W.block_hierarchy(mesh.grid_shape, (f,) * dim, 3)
    disc = sipg.assemble(mesh.vertices, mesh.elements, D, p, 1, 0.0)
    inherited = mg.build_hierarchy(disc, 20.0, maps)
    direct = mg.build_hierarchy(disc, 20.0, maps, direct=dict(D=D, c_pen=0.0))
    for l in (1, 2):
        a, b = direct.levels[l].A, inherited.levels[l].A
        assert abs(a - b).max() <= 1e-13 * abs(b).max(), l


def test_jittered_levels_are_symmetric_with_constants_in_the_kernel():
    wl = W.jittered_square_2d(n=16, degree=2, n_levels=3)
    disc = sipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, 2, 1, 4.0)
    lo, hi = mg.level1_boxes(disc.vertices, disc.elements, np.asarray(wl.maps[0], np.int64))
    unit = np.asarray(wl.maps[0], np.int64)
    for l in range(2):
        A = dc.level_operator(disc.vertices, disc.elements, wl.conductivity, 2, 0.0, 16.0, unit, lo, hi).toarray()
        scale = np.abs(A).max()
        assert np.abs(A - A.T).max() <= 1e-14 * scale
        assert np.abs(A @ np.ones(A.shape[0])).max() <= 1e-13 * scale
        ev = np.linalg.eigvalsh(A)
        assert ev.min() >= -1e-12 * scale
        assert np.sum(ev < 1e-12 * scale) == 1
        if l == 0:
            amap = np.asarray(wl.maps[1], np.int64)
            lo, hi = mg.coarser_boxes(lo, hi, amap)
            unit = amap[unit]
