"""The non-inherited coarse operators (agg_mg_opts.coarse_operator = 1,
Section 5.1) on the device against the oracle's hierarchy built with them
(oracle/direct_coarse.py), float64 form: every level's operator, one
V-cycle, and PCG iterations and solution. The float32 form runs the same
hierarchy and reaches the same residual."""
import numpy as np
import pytest

from oracle import multigrid as omg
from oracle import sipg as osipg
from paper_2602_16312_gb300 import workloads as W

from gpu_util import rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_16312_gb300 import build
    build.build()


CASES = {
    "jsquare2d_q2_30": lambda: W.jittered_square_2d(n=30, n_levels=3),
    "jcube3d_q2_6": lambda: W.jittered_cube_3d(n=6, degree=2, n_levels=3, group=2),
    "shell_q2": lambda: W.ventricle_shell(16, 8, 4, n_levels=3),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    from paper_2602_16312_gb300 import aggmg
    wl = CASES[request.param]()
    disc = osipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, wl.degree,
                          wl.penalty_mode, wl.penalty_coeff)
    c_pen = osipg.penalty_constant(wl.degree, wl.penalty_mode, wl.penalty_coeff)
    c = 1.0 / wl.dt
    ho = omg.build_hierarchy(disc, c, wl.maps, direct=dict(D=wl.conductivity, c_pen=c_pen))
    mesh = aggmg.Mesh.from_workload(wl)
    hier = aggmg.Hierarchy(mesh, c, wl.maps, precision="f64", coarse_operator="direct")
    return wl, disc, ho, mesh, hier


def _dev(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda")


def test_direct_operator_apply_every_level(case):
    wl, disc, ho, mesh, hier = case
    rng = np.random.default_rng(21)
    for l, lev in enumerate(ho.levels[:-1]):
        x = rng.standard_normal(lev.A.shape[0])
        y = torch.empty(lev.A.shape[0], dtype=torch.float64, device="cuda")
        hier.operator_apply(l, _dev(x), y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), lev.A @ x) <= 1e-13, l


def test_direct_vcycle_and_pcg_match_oracle(case):
    wl, disc, ho, mesh, hier = case
    rng = np.random.default_rng(22)
    r = rng.standard_normal(disc.n)
    z = torch.empty(disc.n, dtype=torch.float64, device="cuda")
    hier.vcycle_apply(_dev(r), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), omg.vcycle(ho, r)) <= 1e-11
    b = rng.standard_normal(disc.n)
    x0 = rng.standard_normal(disc.n)
    ref = omg.pcg(ho.levels[0].A, b, x0, lambda v: omg.vcycle(ho, v), rtol=1e-10)
    x = _dev(x0)
    res = hier.pcg_solve(_dev(b), x, rtol=1e-10)
    assert res["iterations"] == ref.iterations
    assert rel(x.cpu().numpy(), ref.x) <= 1e-10


def test_direct_f32_form_converges_like_f64(case):
    from paper_2602_16312_gb300 import aggmg
    wl, disc, ho, mesh, hier = case
    h32 = aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps, precision="f32", coarse_operator="direct")
    rng = np.random.default_rng(23)
    b = rng.standard_normal(disc.n)
    ref = omg.pcg(ho.levels[0].A, b, np.zeros(disc.n), lambda v: omg.vcycle(ho, v), rtol=1e-8)
    x = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    res = h32.pcg_solve(_dev(b), x, rtol=1e-8, flexible=True)
    assert abs(res["iterations"] - ref.iterations) <= 1
    r = b - ho.levels[0].A @ x.cpu().numpy()
    assert np.linalg.norm(r) <= 1.05e-8 * np.linalg.norm(b)
