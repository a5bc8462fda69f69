"""CUDA path against the oracle, element by element (float64 form), through
the C ABI. Sizes span several 32-unit slices with a ragged tail."""
import numpy as np
import pytest

from oracle import monodomain as omd
from oracle import multigrid as omg
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


def _aggmg():
    from paper_2602_16312_gb300 import aggmg
    return aggmg


CASES = {
    "square2d_q1_16": lambda: W.square_2d_fhn(16, 1),
    "jsquare2d_q2_30": lambda: W.jittered_square_2d(n=30, n_levels=3),
    "jcube3d_q1_6": lambda: W.jittered_cube_3d(n=6, degree=1, n_levels=3, group=2),
    "jcube3d_q2_6": lambda: W.jittered_cube_3d(n=6, degree=2, n_levels=3, group=2),
    "shell_q2": lambda: W.ventricle_shell(16, 8, 4, n_levels=3),
    "jcube3d_q3_6": lambda: W.jittered_cube_3d(n=6, degree=3, n_levels=3, group=2),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    aggmg = _aggmg()
    wl = CASES[request.param]()
    disc, ho = oracle_setup(wl)
    mesh = aggmg.Mesh.from_workload(wl)
    hier = aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps, precision="f64")
    return wl, disc, ho, mesh, hier


def _dev(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda")


def test_operator_apply_every_level(case):
    wl, disc, ho, mesh, hier = case
    rng = np.random.default_rng(11)
    for l, lev in enumerate(ho.levels[:-1]):
        x = rng.standard_normal(lev.A.shape[0])
        y = torch.empty(lev.A.shape[0], dtype=torch.float64, device="cuda")
        hier.operator_apply(l, _dev(x), y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), lev.A @ x) <= 1e-13, l


def test_vcycle_matches_oracle(case):
    wl, disc, ho, mesh, hier = case
    r = np.random.default_rng(12).standard_normal(disc.n)
    z = torch.empty(disc.n, dtype=torch.float64, device="cuda")
    hier.vcycle_apply(_dev(r), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), omg.vcycle(ho, r)) <= 1e-11


def test_pcg_matches_oracle_iterations_and_solution(case):
    wl, disc, ho, mesh, hier = case
    rng = np.random.default_rng(13)
    b = rng.standard_normal(disc.n)
    x0 = rng.standard_normal(disc.n)
    ref = omg.pcg(ho.levels[0].A, b, x0, lambda r: omg.vcycle(ho, r), rtol=1e-10)
    x = _dev(x0)
    res = hier.pcg_solve(_dev(b), x, rtol=1e-10)
    assert res["iterations"] == ref.iterations
    assert abs(res["r0_norm"] - ref.r0_norm) <= 1e-12 * ref.r0_norm
    assert rel(x.cpu().numpy(), ref.x) <= 1e-10


def test_monodomain_trajectory_matches_oracle(case):
    aggmg = _aggmg()
    wl, disc, ho, mesh, hier = case
    n_steps = 8
    opts = step_opts(wl)
    mask = wl.stim_mask_nodal()
    u_ref, w_ref, its_ref = omd.run(disc, ho, opts, np.zeros(disc.n), np.zeros(disc.n), mask, n_steps)
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(mask), iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol)
    u = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    its = sim.step(u, w, n_steps)
    sim.close()
    assert its == its_ref
    assert rel(u.cpu().numpy(), u_ref) <= 1e-10
    assert rel(w.cpu().numpy(), w_ref) <= 1e-10


def test_ionic_update_matches_oracle():
    aggmg = _aggmg()
    rng = np.random.default_rng(14)
    u = rng.uniform(-0.1, 1.1, 1000)
    w = rng.uniform(0, 1.5, 1000)
    for prm in (W.FHN, W.ALIEV_PANFILOV):
        wd = _dev(w)
        aggmg.ionic_update(prm, 0.05, _dev(u), wd)
        torch.cuda.synchronize()
        _, H = omd.ionic(prm, u, w)
        assert rel(wd.cpu().numpy(), w + 0.05 * H) <= 1e-15


def test_error_statuses():
    aggmg = _aggmg()
    wl = W.square_2d_fhn(8, 1)
    disc, ho = oracle_setup(wl)
    mesh = aggmg.Mesh.from_workload(wl)
    hier = aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps)
    b = np.random.default_rng(15).standard_normal(disc.n)
    res = hier.pcg_solve(_dev(b), _dev(np.zeros(disc.n)), rtol=1e-12, max_it=1, check=False)
    assert res["status"] == aggmg.AGG_ENOTCONV and res["iterations"] == 1
    b[3] = np.nan
    res = hier.pcg_solve(_dev(b), _dev(np.zeros(disc.n)), rtol=1e-12, check=False)
    assert res["status"] == aggmg.AGG_ENAN
    # zero right-hand side and zero guess: converged before the first iteration
    res = hier.pcg_solve(_dev(np.zeros(disc.n)), _dev(np.zeros(disc.n)))
    assert res["iterations"] == 0 and res["status"] == 0


@pytest.mark.parametrize("name", ["square2d_q1_16", "jsquare2d_q2_30", "jcube3d_q2_6"])
def test_bdf2_trajectory_matches_oracle(name):
    """Scheme 1 (BDF2 with extrapolation and the derivative start) against the
    oracle's BDF2: same iteration counts, states within 1e-10."""
    aggmg = _aggmg()
    wl = CASES[name]()
    c = 1.5 / wl.dt
    disc, ho = oracle_setup(wl, c=c)
    opts = step_opts(wl)
    opts.scheme = 1
    mask = wl.stim_mask_nodal()
    n_steps = 8
    u_ref, w_ref, its_ref = omd.run(disc, ho, opts, np.zeros(disc.n), np.zeros(disc.n), mask, n_steps)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), c, wl.maps, precision="f64")
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(mask), iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol, scheme=1)
    u = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    its = sim.step(u, w, 3) + sim.step(u, w, n_steps - 3)     # history carried across calls
    sim.close()
    assert its == its_ref
    assert rel(u.cpu().numpy(), u_ref) <= 1e-10
    assert rel(w.cpu().numpy(), w_ref) <= 1e-10
    # the mass coefficient must match the scheme
    with pytest.raises(aggmg.AggError):
        aggmg.Monodomain(hier, wl.dt, wl.ionic, scheme=0)


def test_plain_fp64_square_all_fifty_steps_match_oracle_every_step():
    """The 16x16 Q1 square as configured (plain float64, 2 levels of 4x4
    agglomerates, rtol 1e-10, FitzHugh-Nagumo, stimulus for 5 steps, 50
    steps from rest): after every step, the same PCG iteration count as the
    oracle and u, w within 1e-10 of the oracle's largest entry."""
    aggmg = _aggmg()
    wl = W.square_2d_fhn(16, 1)
    assert wl.n_steps == 50 and wl.rtol == 1e-10
    disc, ho = oracle_setup(wl)
    opts = step_opts(wl)
    mask = wl.stim_mask_nodal()
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f64")
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(mask), iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol)
    u = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    uo, wo = np.zeros(disc.n), np.zeros(disc.n)
    for n in range(wl.n_steps):
        its = sim.step(u, w, 1)
        uo, wo, res = omd.step(disc, ho, opts, uo, wo, mask, n)
        assert its[0] == res.iterations, (n, its, res.iterations)
        assert rel(u.cpu().numpy(), uo) <= 1e-10, (n, worst(u.cpu().numpy(), uo))
        assert rel(w.cpu().numpy(), wo) <= 1e-10, (n, worst(w.cpu().numpy(), wo))
    sim.close()
    hier.close()
