"""Matrix-free fine operator (float32; quadrilaterals and hexahedra) of the
V-cycle against the oracle's assembled float64 operator, and the solver built
on it against the float64 oracle (the float32 V-cycle tolerance and the 1e-8
trajectory bound)."""
import dataclasses

import numpy as np
import pytest

from oracle import monodomain as omd
from oracle import multigrid as omg
from paper_2602_16312_gb300 import workloads as W

from gpu_util import oracle_setup, rel, step_opts

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_16312_gb300 import build
    build.build()


def _dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


CASES = {
    "jsquare2d_q1_30": lambda: W.jittered_square_2d(n=30, degree=1, n_levels=3),
    "jsquare2d_q2_30": lambda: W.jittered_square_2d(n=30, degree=2, n_levels=3),
    "jsquare2d_q3_18": lambda: W.jittered_square_2d(n=18, degree=3, n_levels=2),
    "square2d_q1_16": lambda: W.square_2d_fhn(16, 1),
    "jcube3d_q1_6": lambda: W.jittered_cube_3d(n=6, degree=1, n_levels=3, group=2),
    "jcube3d_q2_6": lambda: W.jittered_cube_3d(n=6, degree=2, n_levels=3, group=2),
    "shell_q2": lambda: W.ventricle_shell(16, 8, 4, n_levels=3),
}
# hexahedra of p = 3 (64 DoFs per element): the float32 operator only
CASES_F32 = dict(CASES, jcube3d_q3_4=lambda: W.jittered_cube_3d(n=4, degree=3, n_levels=2, group=2),
                 cube3d_q3_4=lambda: W.cube_3d_adjoint(n=4, n_levels=3))


def _rotated_element_cube():
    """6^3 jittered Q2 cube whose element 0 lists its corners rotated by 90
    degrees about the z axis: a valid mesh whose shared faces of element 0
    are parametrised differently by the two sides."""
    wl = W.jittered_cube_3d(n=6, degree=2, n_levels=3, group=2)
    el = wl.mesh.elements.copy()
    old = el[0].copy()
    for c in range(8):
        i, j, k = c & 1, (c >> 1) & 1, (c >> 2) & 1
        el[0, c] = old[(1 - j) | (i << 1) | (k << 2)]
    return dataclasses.replace(wl, mesh=dataclasses.replace(wl.mesh, elements=el))


@pytest.mark.parametrize("name", list(CASES_F32))
def test_matrix_free_operator_matches_assembled(name):
    from paper_2602_16312_gb300 import aggmg
    wl = CASES_F32[name]()
    disc, ho = oracle_setup(wl)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f32", fine="mf")
    x = np.random.default_rng(51).standard_normal(disc.n)
    y = torch.empty(disc.n, dtype=torch.float64, device="cuda")
    hier.operator_apply(-1, _dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ho.levels[0].A @ x) <= 2e-6


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("form", ["f64", "f32"])
def test_float64_matrix_free_operator_matches_assembled(name, form):
    """The float64 matrix-free level-0 operator (agg_operator_apply level -2,
    the measured alternative for the outer CG) against the oracle's assembled
    A0, in a hierarchy of either V-cycle precision."""
    from paper_2602_16312_gb300 import aggmg
    wl = CASES[name]()
    disc, ho = oracle_setup(wl)
    fine = "mf" if form == "f32" else "bsr"
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision=form, fine=fine)
    x = np.random.default_rng(52).standard_normal(disc.n)
    y = torch.empty(disc.n, dtype=torch.float64, device="cuda")
    for _ in range(2):                     # first call builds the data
        hier.operator_apply(-2, _dev(x), y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), ho.levels[0].A @ x) <= 1e-12
    b, f = hier.kernel_cost(5)
    b0, f0 = hier.kernel_cost(0)
    assert b > 0 and f == f0
    hier.profile_kernel(5, 2)
    torch.cuda.synchronize()
    hier.close()


@pytest.mark.parametrize("name", list(CASES_F32))
def test_matrix_free_vcycle_and_trajectory(name):
    from paper_2602_16312_gb300 import aggmg
    wl = CASES_F32[name]()
    disc, ho = oracle_setup(wl)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f32", fine="mf")
    r = np.random.default_rng(52).standard_normal(disc.n)
    z = torch.empty(disc.n, dtype=torch.float64, device="cuda")
    hier.vcycle_apply(_dev(r), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), omg.vcycle(ho, r)) <= 5e-6
    opts = step_opts(wl)
    mask = wl.stim_mask_nodal()
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(mask), iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol, flexible=True)
    u = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    uo, wo = np.zeros(disc.n), np.zeros(disc.n)
    for n in range(5):
        uo, wo, res = omd.step(disc, ho, opts, uo, wo, mask, n)
        its = sim.step(u, w, 1)
        assert rel(u.cpu().numpy(), uo) <= 1e-8, n
        assert abs(its[0] - res.iterations) <= 3
    sim.close()


def test_matrix_free_rejected_where_unsupported():
    from paper_2602_16312_gb300 import aggmg
    # the float64 matrix-free operator is built for hexahedra of p <= 2 only
    wl = W.jittered_cube_3d(n=4, degree=3, n_levels=2, group=2)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f64")
    x = torch.zeros(wl.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(aggmg.AggError) as e:
        hier.operator_apply(-2, x, torch.empty_like(x))
    assert e.value.status == aggmg.AGG_EUNSUPPORTED
    hier.close()
    # shared faces parametrised differently by the two sides: the assembled
    # operator takes the mesh, the 3D matrix-free one reports it unsupported
    wl = _rotated_element_cube()
    mesh = aggmg.Mesh.from_workload(wl)
    aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps, precision="f32").close()
    with pytest.raises(aggmg.AggError) as e:
        aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps, precision="f32", fine="mf")
    assert e.value.status == aggmg.AGG_EUNSUPPORTED
    wl = W.jittered_square_2d(n=8, degree=2, n_levels=2)
    with pytest.raises(aggmg.AggError) as e:
        aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f64", fine="mf")
    assert e.value.status == aggmg.AGG_EUNSUPPORTED
