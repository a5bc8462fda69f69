"""Adjoint form on the GPU: reverse steps against the oracle's adjoint, and
the conductivity gradient of a sensor loss against the oracle's FP64 adjoint
and against central differences of GPU forward runs."""
import numpy as np
import pytest

from oracle import monodomain as omd
from oracle import sipg as osipg
from paper_2602_16312_gb300 import workloads as W

from gpu_util import oracle_setup, rel, step_opts, worst

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
    "jsquare2d_q2_12": lambda: W.jittered_square_2d(n=12, n_levels=2),
    "jcube3d_q1_6": lambda: W.jittered_cube_3d(n=6, degree=1, n_levels=3, group=2),
    "jcube3d_q2_4": lambda: W.jittered_cube_3d(n=4, degree=2, n_levels=2, group=2),
    "cube3d_q3_4": lambda: W.cube_3d_adjoint(n=4, degree=3, n_levels=2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_step_matches_oracle(name):
    from paper_2602_16312_gb300 import aggmg
    wl = CASES[name]()
    disc, ho = oracle_setup(wl)
    forms = osipg.attributed_forms(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, wl.degree,
                                   wl.penalty_mode, wl.penalty_coeff)
    opts = step_opts(wl, rtol=1e-12)
    rng = np.random.default_rng(31)
    u_n = rng.uniform(0, 0.8, disc.n)
    w_n = rng.uniform(0, 0.5, disc.n)
    u_np1 = u_n + 0.01 * rng.standard_normal(disc.n)
    ubar = rng.standard_normal(disc.n)
    wbar = rng.standard_normal(disc.n)
    ub_o, wb_o, g_o = omd.adjoint_step(disc, ho, opts, forms, u_n, w_n, u_np1, ubar, wbar, rtol=1e-12)
    mesh = aggmg.Mesh.from_workload(wl, adjoint_data=True)
    hier = aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps, precision="f64")
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, rtol=1e-12)
    ub, wb = _dev(ubar), _dev(wbar)
    g = torch.zeros(wl.mesh.n_elements, dtype=torch.float64, device="cuda")
    sim.adjoint_step(_dev(u_n), _dev(w_n), _dev(u_np1), ub, wb, g)
    assert rel(ub.cpu().numpy(), ub_o) <= 1e-9
    assert rel(wb.cpu().numpy(), wb_o) <= 1e-9
    assert rel(g.cpu().numpy(), g_o) <= 1e-9
    sim.close()


def _problem(form="f64", n=6):
    wl = W.jittered_square_2d(n=n, degree=1, n_levels=2)
    wl.maps = W.block_hierarchy(wl.mesh.grid_shape, (2, 2), 2)
    wl.conductivity = W.conductivity_from_fibres(W.planar_fibres(wl.mesh.n_elements, 30.0), 1.2e-2, 2.5e-3)
    wl.ionic = dict(W.ALIEV_PANFILOV, eps=0.02)
    wl.iapp_steps = 3
    tmap, tshape = W.block_map(wl.mesh.grid_shape, (3, 3))
    theta = np.exp(0.2 * np.random.default_rng(41).standard_normal(int(np.prod(tshape))))
    return wl, tmap, theta


def _loss(problem, sensors, target, theta, n_steps, K=2):
    from paper_2602_16312_gb300.autograd import MonodomainRun
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    z = torch.zeros(problem.n_dofs, dtype=torch.float64, device="cuda")
    u, w = MonodomainRun.apply(th, z, z.clone(), problem, n_steps, K)
    val = problem.evaluate(u, sensors)
    return ((val - target) ** 2).sum(), th


def test_theta_gradient_matches_oracle_adjoint_and_finite_differences():
    from paper_2602_16312_gb300.autograd import MonodomainProblem
    wl, tmap, theta = _problem()
    n_steps = 6
    problem = MonodomainProblem(wl, tmap, precision="f64", rtol=1e-12)
    pts = np.random.default_rng(42).uniform(0.05, 0.95, size=(12, 2))
    problem.build(np.ones_like(theta))
    sensors = problem.sensors(pts)
    # target = sensor values of the theta = 1 run
    from paper_2602_16312_gb300.autograd import MonodomainRun
    z = torch.zeros(problem.n_dofs, dtype=torch.float64, device="cuda")
    u1, _ = MonodomainRun.apply(torch.ones(len(theta), dtype=torch.float64), z, z.clone(), problem, n_steps, 2)
    target = problem.evaluate(u1, sensors).detach()
    L, th = _loss(problem, sensors, target, theta, n_steps)
    L.backward()
    g = th.grad.numpy()
    # oracle FP64 adjoint of the same loss
    D = wl.conductivity * theta[tmap][:, None, None]
    from oracle import multigrid as omg
    disc = osipg.assemble(wl.mesh.vertices, wl.mesh.elements, D, wl.degree, wl.penalty_mode, wl.penalty_coeff)
    ho = omg.build_hierarchy(disc, 1.0 / wl.dt, wl.maps)
    opts = step_opts(wl, rtol=1e-12)
    mask = wl.stim_mask_nodal()
    us, ws = omd.trajectory(disc, ho, opts, np.zeros(disc.n), np.zeros(disc.n), mask, n_steps)
    elem, Wt = osipg.locate_points(wl.mesh.vertices, wl.mesh.elements, wl.degree, pts)
    val = np.einsum("si,si->s", Wt, us[-1].reshape(-1, disc.B)[elem])
    ubar = np.zeros(disc.n)
    np.add.at(ubar.reshape(-1, disc.B), elem, 2 * (val - target.cpu().numpy())[:, None] * Wt)
    forms = osipg.attributed_forms(wl.mesh.vertices, wl.mesh.elements, D, wl.degree, wl.penalty_mode,
                                   wl.penalty_coeff)
    gamma, _, _ = omd.gradient_log_conductivity(disc, ho, opts, forms, us, ws, ubar)
    g_o = np.zeros_like(theta)
    np.add.at(g_o, tmap, gamma)
    g_o /= theta
    assert rel(g, g_o) <= 1e-6, (g, g_o)
    # central differences of GPU forward runs on every component
    for k in range(len(theta)):
        h = 1e-5 * theta[k]
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        with torch.no_grad():
            Lp, _ = _loss(problem, sensors, target, tp, n_steps)
            Lm, _ = _loss(problem, sensors, target, tm, n_steps)
        fd = (Lp.item() - Lm.item()) / (2 * h)
        assert abs(g[k] - fd) <= 1e-5 * np.abs(g).max(), (k, g[k], fd)


def test_theta_gradient_reduction_matches_the_chain_rule():
    """agg_theta_gradient: sum of per-element log-conductivity gradients over
    each parameter's elements, divided by theta, accumulated."""
    from paper_2602_16312_gb300 import aggmg
    wl = W.jittered_square_2d(n=12, degree=1, n_levels=2)
    tmap, tshape = W.block_map(wl.mesh.grid_shape, (3, 2))
    theta = np.exp(0.2 * np.random.default_rng(5).standard_normal(int(np.prod(tshape))))
    mesh = aggmg.Mesh.from_workload(wl, theta=theta, theta_map=tmap)
    hier = aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps)
    g = np.random.default_rng(6).standard_normal(wl.mesh.n_elements)
    out0 = np.random.default_rng(7).standard_normal(len(theta))
    out = torch.tensor(out0, device="cuda")
    hier.theta_gradient(torch.tensor(g, device="cuda"), out)
    ref = out0.copy()
    np.add.at(ref, tmap, g)
    ref = out0 + (ref - out0) / theta
    assert rel(out.cpu().numpy(), ref) <= 1e-14
    hier.close()


def test_theta_gradient_q3_hexahedra_with_sensors_and_checkpoints():
    """The adjoint workload's form at a size the oracle solves: DG Q3 on
    hexahedra, float64, conductivity scales theta on 2x2x2 element blocks
    (lognormal, sigma 0.2), Aliev-Panfilov, squared error at seeded sensor
    points against the theta = 1 run, checkpoints every 2 of 6 steps. The
    gradient against the oracle's float64 adjoint and against central
    differences of GPU forward runs on 8 seeded components, 1e-6 relative."""
    from paper_2602_16312_gb300.autograd import MonodomainProblem, MonodomainRun
    wl = W.cube_3d_adjoint(n=6, n_levels=3)
    wl.maps = W.block_hierarchy(wl.mesh.grid_shape, (2, 2, 2), 3)
    tmap, tshape = W.block_map(wl.mesh.grid_shape, (2, 2, 2))
    rng = np.random.default_rng(3)
    theta = np.exp(0.2 * rng.standard_normal(int(np.prod(tshape))))
    pts = rng.uniform(0.0, 1.0, size=(64, 3))
    comps = rng.choice(len(theta), 8, replace=False)
    n_steps, K = 6, 2
    problem = MonodomainProblem(wl, tmap, precision="f64", rtol=1e-12)
    problem.build(np.ones_like(theta))
    sensors = problem.sensors(pts)
    z = torch.zeros(problem.n_dofs, dtype=torch.float64, device="cuda")
    u1, _ = MonodomainRun.apply(torch.ones(len(theta), dtype=torch.float64), z, z.clone(), problem, n_steps, K)
    target = problem.evaluate(u1, sensors).detach()
    L, th = _loss(problem, sensors, target, theta, n_steps, K)
    L.backward()
    g = th.grad.numpy()
    # oracle float64 adjoint
    from oracle import multigrid as omg
    D = wl.conductivity * theta[tmap][:, None, None]
    disc = osipg.assemble(wl.mesh.vertices, wl.mesh.elements, D, wl.degree, wl.penalty_mode, wl.penalty_coeff)
    ho = omg.build_hierarchy(disc, 1.0 / wl.dt, wl.maps)
    opts = step_opts(wl, rtol=1e-12)
    mask = wl.stim_mask_nodal()
    us, ws = omd.trajectory(disc, ho, opts, np.zeros(disc.n), np.zeros(disc.n), mask, n_steps)
    elem, Wt = osipg.locate_points(wl.mesh.vertices, wl.mesh.elements, wl.degree, pts)
    val = np.einsum("si,si->s", Wt, us[-1].reshape(-1, disc.B)[elem])
    ubar = np.zeros(disc.n)
    np.add.at(ubar.reshape(-1, disc.B), elem, 2 * (val - target.cpu().numpy())[:, None] * Wt)
    forms = osipg.attributed_forms(wl.mesh.vertices, wl.mesh.elements, D, wl.degree, wl.penalty_mode,
                                   wl.penalty_coeff)
    gamma, _, _ = omd.gradient_log_conductivity(disc, ho, opts, forms, us, ws, ubar)
    g_o = np.zeros_like(theta)
    np.add.at(g_o, tmap, gamma)
    g_o /= theta
    assert rel(g, g_o) <= 1e-6, worst(g, g_o)
    for k in comps:
        h = 1e-5 * theta[k]
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        with torch.no_grad():
            Lp, _ = _loss(problem, sensors, target, tp, n_steps, K)
            Lm, _ = _loss(problem, sensors, target, tm, n_steps, K)
        fd = (Lp.item() - Lm.item()) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * abs(g[k]) + 1e-9 * np.abs(g).max(), (k, g[k], fd)
