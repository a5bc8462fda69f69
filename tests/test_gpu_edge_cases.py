"""Degenerate and empty cases of the CUDA path through the C ABI: a
single-level hierarchy (the V-cycle is the coarsest Cholesky solve, so PCG
converges in one iteration), a mesh of one element (no interior face), empty
updates and zero-step calls."""
import numpy as np
import pytest

from oracle import multigrid as omg
from paper_2602_16312_gb300 import workloads as W

from gpu_util import oracle_setup, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_16312_gb300 import build
    build.build()


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision,fine", [("f64", "bsr"), ("f32", "mf"), ("f32", "bsr")])
def test_single_level_hierarchy_is_a_direct_solve(precision, fine):
    from paper_2602_16312_gb300 import aggmg
    wl = W.jittered_square_2d(n=10, degree=2, n_levels=2)
    wl.maps = []
    disc, ho = oracle_setup(wl)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision=precision, fine=fine)
    assert hier.n_levels == 1
    b = np.random.default_rng(71).standard_normal(disc.n)
    z = torch.empty(disc.n, dtype=torch.float64, device="cuda")
    hier.vcycle_apply(_dev(b), z)
    torch.cuda.synchronize()
    x_direct = omg.vcycle(ho, b)                     # one level: the Cholesky solve
    tol = 1e-12 if precision == "f64" else 1e-4              # float32 input rounding times cond(A0)
    assert rel(z.cpu().numpy(), x_direct) <= tol
    x = _dev(np.zeros(disc.n))
    res = hier.pcg_solve(_dev(b), x, rtol=1e-6 if precision != "f64" else 1e-10, flexible=precision != "f64")
    assert res["iterations"] <= (1 if precision == "f64" else 3)
    hier.close()


@pytest.mark.parametrize("dim,degree", [(2, 2), (3, 1), (3, 2)])
def test_one_element_mesh(dim, degree):
    """No interior face: the operator is the element's c M_e + K_e, the
    hierarchy has one level, and a time step solves it directly."""
    from paper_2602_16312_gb300 import aggmg
    mesh = W.box_mesh(dim, 1)
    D = W.conductivity_from_fibres(W.planar_fibres(1, 30.0) if dim == 2 else W.rotating_fibres_z(mesh.centroids()),
                                   1.2e-3, 2.5e-4)
    wl = W.Workload(name="one", mesh=mesh, degree=degree, conductivity=D, maps=[], penalty_mode=1,
                    penalty_coeff=10.0, dt=0.05, n_steps=1, ionic=dict(W.FHN),
                    stim_elements=np.ones(1, dtype=bool), iapp_value=1.0, iapp_steps=5, rtol=1e-10)
    disc, ho = oracle_setup(wl)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f64")
    x = np.random.default_rng(72).standard_normal(disc.n)
    y = torch.empty(disc.n, dtype=torch.float64, device="cuda")
    hier.operator_apply(0, _dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ho.levels[0].A @ x) <= 1e-13
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(wl.stim_mask_nodal()), iapp_value=1.0,
                           iapp_steps=5, rtol=1e-10)
    u = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    its = sim.step(u, w, 2)
    assert all(i <= 1 for i in its) and torch.isfinite(u).all()
    # the uniform stimulus on the only element raises u uniformly
    assert u.min().item() > 0
    sim.close()
    hier.close()


def test_empty_and_zero_step_calls():
    from paper_2602_16312_gb300 import aggmg
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    for prm in (W.FHN, W.BUENO_OROVIO):
        aggmg.ionic_update(prm, 0.05, e, e)                   # n = 0: nothing to do, no error
    wl = W.square_2d_fhn(8, 1)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps)
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic)
    u0 = torch.rand(wl.n_dofs, dtype=torch.float64, device="cuda")
    w0 = torch.rand(wl.n_dofs, dtype=torch.float64, device="cuda")
    u, w = u0.clone(), w0.clone()
    assert sim.step(u, w, 0) == []                            # zero steps leave the state as it is
    assert torch.equal(u, u0) and torch.equal(w, w0)
    with pytest.raises(aggmg.AggError) as err:
        sim.step(u, w, -1, iters=False)
    assert err.value.status == aggmg.AGG_EINVAL
    sim.close()
    hier.close()
