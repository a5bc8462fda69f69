"""The library's non-inherited coarse operators (HierOptions::direct,
agg_mg_opts.coarse_operator = 1; Section 5.1) against the oracle's
(oracle/direct_coarse.py), on the CPU through the host inspection entry
points: every block of every coarse level, the smoother blocks and the
Chebyshev bounds computed from them."""
import numpy as np
import pytest

from oracle import multigrid as omg
from oracle import sipg as osipg
from paper_2602_16312_gb300 import aggmg
from paper_2602_16312_gb300 import workloads as W

from test_host_setup import _bsr_to_csr


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2602_16312_gb300 import build
    build.build()


CASES = {
    "square2d_q1": lambda: W.square_2d_fhn(16, 1),
    "jsquare2d_q2": lambda: W.jittered_square_2d(n=16, n_levels=3),
    "jcube3d_q2": lambda: W.jittered_cube_3d(n=4, degree=2, n_levels=3, group=2),
    "shell_q2": lambda: W.ventricle_shell(16, 8, 4, n_levels=3),
    "cube3d_q3": lambda: W.cube_3d_adjoint(n=4, degree=3, n_levels=2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_direct_coarse_levels_match_oracle(name):
    wl = CASES[name]()
    disc = osipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, wl.degree,
                          wl.penalty_mode, wl.penalty_coeff)
    c_pen = osipg.penalty_constant(wl.degree, wl.penalty_mode, wl.penalty_coeff)
    c = 1.0 / wl.dt
    ho = omg.build_hierarchy(disc, c, wl.maps, direct=dict(D=wl.conductivity, c_pen=c_pen))
    mesh = aggmg.Mesh.from_workload(wl)
    hh = aggmg.HostHierarchy(mesh, c, wl.maps, coarse_operator="direct")
    inherited = aggmg.HostHierarchy(mesh, c, wl.maps)
    for l, lev in enumerate(ho.levels):
        n, nnzb, lam = hh.level(l)
        assert n == lev.n_units
        perm = hh.copy(l, 0)
        Al = _bsr_to_csr(hh.copy(l, 1), hh.copy(l, 2), hh.copy(l, 3), n, n, perm)
        scale = abs(lev.A).max()
        assert abs(Al - lev.A).max() <= 1e-12 * scale, l
        if l < len(ho.levels) - 1:
            Dinv = hh.copy(l, 4)
            np.testing.assert_allclose(Dinv, lev.Dinv[perm], rtol=0, atol=1e-10 * np.abs(lev.Dinv).max())
            assert abs(lam - lev.lam_max) <= 1e-10 * lev.lam_max
        if l >= 1 and n > 1:
            # not the Galerkin product: the coarse penalty differs wherever
            # agglomerates meet (one agglomerate alone differs only by the
            # box basis not being in the fine space of a jittered mesh)
            Ai = _bsr_to_csr(inherited.copy(l, 1), inherited.copy(l, 2), inherited.copy(l, 3), n, n,
                             inherited.copy(l, 0))
            assert abs(Ai - Al).max() > 1e-6 * scale, l


def test_unknown_coarse_operator_is_rejected():
    wl = W.square_2d_fhn(8, 1)
    mesh = aggmg.Mesh.from_workload(wl)
    with pytest.raises(aggmg.AggError):
        aggmg.HostHierarchy(mesh, 20.0, wl.maps, coarse_operator=2)
