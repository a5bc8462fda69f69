"""The library's host float64 set-up (assembly and Algorithm 3) against the
oracle, on the CPU through the C ABI's host inspection entry points."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import multigrid as omg
from oracle import sipg as osipg
from paper_2602_16312_gb300 import aggmg
from paper_2602_16312_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    """The host set-up runs in libaggmg.so: build it (nvcc cross-compiles
    without a GPU) if this checkout has no current build."""
    from paper_2602_16312_gb300 import build
    build.build()


def _bsr_to_csr(rp, cols, vals, n_rows, n_cols, perm=None):
    B = vals.shape[1]
    rows = np.repeat(np.arange(n_rows), np.diff(rp))
    c = cols.astype(np.int64)
    if perm is not None:
        rows, c = perm[rows], perm[c]
    m = sp.bsr_matrix((vals, c, np.arange(len(c) + 1)), shape=(len(c) * B, n_cols * B))
    # assemble block rows explicitly (bsr with one block per "row" then sum)
    ii, jj = np.meshgrid(np.arange(B), np.arange(B), indexing="ij")
    R = (rows[:, None, None] * B + ii).ravel()
    Cc = (c[:, None, None] * B + jj).ravel()
    del m
    return sp.csr_matrix((vals.ravel(), (R, Cc)), shape=(n_rows * B, n_cols * B))


CASES = {
    "square2d_q1": lambda: W.square_2d_fhn(16, 1),
    "jsquare2d_q2": lambda: W.jittered_square_2d(n=16, n_levels=3),
    "jcube3d_q1": lambda: W.jittered_cube_3d(n=4, degree=1, n_levels=2, group=2),
    "jcube3d_q2": lambda: W.jittered_cube_3d(n=4, degree=2, n_levels=3, group=2),
    "shell_q2": lambda: W.ventricle_shell(16, 8, 4, n_levels=3),
    "cube3d_q3": lambda: W.cube_3d_adjoint(n=4, degree=3, n_levels=2),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    wl = CASES[request.param]()
    disc = osipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, wl.degree,
                          wl.penalty_mode, wl.penalty_coeff)
    mesh = aggmg.Mesh.from_workload(wl)
    return wl, disc, mesh


def test_library_exports_every_declared_symbol():
    import re
    import os
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "aggmg.h")).read()
    declared = set(re.findall(r"\b(agg_[a-z0-9_]+)\s*\(", hdr))
    L = aggmg.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert set(aggmg.exported_symbols()) <= declared | {"agg_mg_opts_default"}


def test_stiffness_mass_volumes_match_oracle(case):
    wl, disc, mesh = case
    rp, cols, vals = mesh.stiffness_bsr()
    A = _bsr_to_csr(rp, cols, vals, mesh.n_elements, mesh.n_elements)
    scale = abs(disc.A).max()
    assert abs(A - disc.A).max() <= 1e-12 * scale
    np.testing.assert_allclose(mesh.element_mass(), disc.Me, rtol=0, atol=1e-14 * np.abs(disc.Me).max())
    np.testing.assert_allclose(mesh.volumes(), disc.volumes, rtol=1e-13)
    nd, nf = mesh.info()
    assert nd == disc.n
    assert nf == len(osipg.find_faces(wl.mesh.elements, wl.mesh.dim)[0])


def test_hierarchy_matches_oracle(case):
    wl, disc, mesh = case
    c = 1.0 / wl.dt
    ho = omg.build_hierarchy(disc, c, wl.maps)
    hh = aggmg.HostHierarchy(mesh, c, wl.maps)
    B = disc.B
    for l, lev in enumerate(ho.levels):
        n, nnzb, lam = hh.level(l)
        assert n == lev.n_units
        perm = hh.copy(l, 0)
        assert sorted(perm.tolist()) == list(range(n))
        Al = _bsr_to_csr(hh.copy(l, 1), hh.copy(l, 2), hh.copy(l, 3), n, n, perm)
        scale = abs(lev.A).max()
        assert abs(Al - lev.A).max() <= 1e-12 * scale, l
        if l < len(ho.levels) - 1:
            Dinv = hh.copy(l, 4)
            np.testing.assert_allclose(Dinv, lev.Dinv[perm], rtol=0, atol=1e-10 * np.abs(lev.Dinv).max())
            assert abs(lam - lev.lam_max) <= 1e-10 * lev.lam_max
            P = hh.copy(l, 5)
            parent = hh.copy(l, 6)
            perm_c = hh.copy(l + 1, 0)
            Po = lev.P.tocsr()
            amap = np.asarray(wl.maps[l])
            assert np.array_equal(perm_c[parent], amap[perm])
            rows = (perm[:, None] * B + np.arange(B)[None, :])          # (n, B)
            colsb = (amap[perm][:, None] * B + np.arange(B)[None, :])    # (n, B)
            Pblk = np.stack([Po[rows[u]][:, colsb[u]].toarray() for u in range(0, n, max(1, n // 64))])
            np.testing.assert_allclose(P[::max(1, n // 64)], Pblk, atol=1e-13)
            # children of every agglomerate are contiguous in the internal order
            assert np.all(np.diff(parent) >= 0)


def test_coupling_blocks_have_exact_face_structure(case):
    """A GLL nodal basis function whose node is off a face vanishes on it, so
    the coupling block of two face neighbours is zero, exactly, outside
    (e's rows on the face) x (all columns) and (all rows) x (n's columns on
    its face). The face-structured device operator stores only those parts."""
    wl, _, mesh = case
    rp, cols, vals = mesh.stiffness_bsr()
    d, B = wl.mesh.dim, mesh.B
    N = round(B ** (1.0 / d))
    idx = np.arange(B)
    on = np.array([(idx // N ** (f // 2)) % N == (f % 2) * (N - 1) for f in range(2 * d)])
    off_both = ~on[:, None, :, None] & ~on[None, :, None, :]          # [f, fn, row, col]
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    blocks = vals[cols != rows]
    assert len(blocks) > 0
    zero = np.all(np.where(off_both[None], blocks[:, None, None], 0.0) == 0.0, axis=(3, 4))
    assert np.all(zero.any(axis=(1, 2)))
    # and the structure is not vacuous: the parts themselves carry nonzeros
    assert np.count_nonzero(blocks) > 0.3 * blocks.size * (1 - ((B - B // N) / B) ** 2)


def test_bad_maps_are_rejected():
    wl = W.square_2d_fhn(8, 1)
    mesh = aggmg.Mesh.from_workload(wl)
    m = np.asarray(wl.maps[0]).copy()
    m[m == 1] = 2                      # id 1 unused
    with pytest.raises(aggmg.AggError) as e:
        aggmg.HostHierarchy(mesh, 20.0, [m])
    assert e.value.status == aggmg.AGG_EINVAL
    m = np.asarray(wl.maps[0]).copy()
    m[0] = -1
    with pytest.raises(aggmg.AggError) as e:
        aggmg.HostHierarchy(mesh, 20.0, [m])
    assert e.value.status == aggmg.AGG_EINVAL


def test_paper_penalty_reported_not_spd():
    """With the paper's C_pen = p(p+1) on the 64x64 jittered anisotropic mesh
    a smoother block is indefinite: set-up fails with AGG_ENOTSPD."""
    wl = W.jittered_square_2d(n=64, n_levels=2)
    mesh = aggmg.Mesh(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, 2, penalty_mode=0)
    with pytest.raises(aggmg.AggError) as e:
        aggmg.HostHierarchy(mesh, 20.0, wl.maps)
    assert e.value.status == aggmg.AGG_ENOTSPD


@pytest.mark.parametrize("dim,p,jit", [(2, 2, 0.2), (3, 1, 0.15)])
def test_adjoint_forms_match_oracle_attribution(dim, p, jit):
    mesh_ = W.box_mesh(dim, 3, jitter=jit, seed=10)
    if dim == 2:
        D = W.conductivity_from_fibres(W.planar_fibres(mesh_.n_elements, 30.0), 1.2e-3, 2.5e-4)
    else:
        D = W.conductivity_from_fibres(W.rotating_fibres_z(mesh_.centroids()), 1.2e-3, 2.5e-4)
    Ke_o, ep, em, Yp, Ym = osipg.attributed_forms(mesh_.vertices, mesh_.elements, D, p, 1, 10.0)
    m = aggmg.Mesh(mesh_.vertices, mesh_.elements, D, p, adjoint_data=True)
    Ke, Y = m.adjoint_forms()
    rp, cols, _ = m.stiffness_bsr()
    scale = np.abs(Yp).max()
    np.testing.assert_allclose(Ke, Ke_o, atol=1e-14 * np.abs(Ke_o).max())
    face_of = {(int(a), int(b)): f for f, (a, b) in enumerate(zip(ep, em))}
    for e in range(mesh_.n_elements):
        for k in range(rp[e], rp[e + 1]):
            n = int(cols[k])
            if n == e:
                assert np.all(Y[k] == 0.0)
                continue
            if e < n:
                f = face_of[(e, n)]
                exp = [Yp[f, 0, 0], Yp[f, 0, 1], Yp[f, 1, 0], Yp[f, 1, 1]]
            else:
                f = face_of[(n, e)]
                exp = [Ym[f, 1, 1], Ym[f, 1, 0], Ym[f, 0, 1], Ym[f, 0, 0]]
            for b in range(4):
                np.testing.assert_allclose(Y[k, b], exp[b], atol=1e-13 * scale)


def test_locate_matches_oracle():
    mesh_ = W.box_mesh(2, 6, jitter=0.2, seed=11)
    D = W.isotropic_conductivity(mesh_.n_elements, 2, 1e-3)
    pts = np.random.default_rng(12).uniform(0, 1, size=(50, 2))
    eo, wo = osipg.locate_points(mesh_.vertices, mesh_.elements, 2, pts)
    m = aggmg.Mesh(mesh_.vertices, mesh_.elements, D, 2)
    el, w = m.locate(pts)
    assert np.array_equal(el, eo)
    np.testing.assert_allclose(w, wo, atol=1e-12)
    with pytest.raises(aggmg.AggError):
        m.locate(np.array([[1.5, 0.5]]))


def test_theta_parameters_scale_the_conductivity():
    """agg_mesh_desc.theta / theta_map: the assembly with theta[map[e]] D_e
    equals, bit for bit, the assembly of the pre-scaled conductivities, and
    bad parameters are rejected."""
    wl = W.jittered_square_2d(n=6, degree=2, n_levels=2)
    tmap, tshape = W.block_map(wl.mesh.grid_shape, (3, 3))
    theta = np.exp(0.2 * np.random.default_rng(3).standard_normal(int(np.prod(tshape))))
    a = aggmg.Mesh.from_workload(wl, theta=theta, theta_map=tmap).stiffness_bsr()
    D = wl.conductivity * theta[tmap][:, None, None]
    b = aggmg.Mesh.from_workload(wl, conductivity=D).stiffness_bsr()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for th, tm in ((-theta, tmap), (theta, tmap + len(theta)), (theta * np.nan, tmap)):
        with pytest.raises(aggmg.AggError) as e:
            aggmg.Mesh.from_workload(wl, theta=th, theta_map=tm)
        assert e.value.status == aggmg.AGG_EINVAL
