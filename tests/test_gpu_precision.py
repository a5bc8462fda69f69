"""Precision forms (float32 V-cycle, bf16-stored smoother blocks) inside the
float64 outer CG: the solution after every solve stays within 1e-8 relative
of the float64 oracle; the V-cycle itself matches the oracle's to float32
accuracy."""
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


CASES = {
    "jsquare2d_q2_30": lambda: W.jittered_square_2d(n=30, n_levels=3),
    "jcube3d_q2_6": lambda: W.jittered_cube_3d(n=6, degree=2, n_levels=3, group=2),
    "jcube3d_q3_6": lambda: W.jittered_cube_3d(n=6, degree=3, n_levels=3, group=2),
}


def _dev(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("form,vtol", [("f32", 3e-6), ("bf16s", 5e-2)])
@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_close_to_oracle(name, form, vtol):
    from paper_2602_16312_gb300 import aggmg
    wl = CASES[name]()
    disc, ho = oracle_setup(wl)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision=form)
    r = np.random.default_rng(21).standard_normal(disc.n)
    z = torch.empty(disc.n, dtype=torch.float64, device="cuda")
    hier.vcycle_apply(_dev(r), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), omg.vcycle(ho, r)) <= vtol


@pytest.mark.parametrize("form", ["f32", "bf16s"])
@pytest.mark.parametrize("name", list(CASES))
def test_trajectory_within_1e8_of_float64_oracle(name, form):
    from paper_2602_16312_gb300 import aggmg
    wl = CASES[name]()
    disc, ho = oracle_setup(wl)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision=form)
    opts = step_opts(wl)
    mask = wl.stim_mask_nodal()
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(mask), iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol, flexible=True)
    u = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    uo, wo = np.zeros(disc.n), np.zeros(disc.n)
    for n in range(6):
        uo, wo, res = omd.step(disc, ho, opts, uo, wo, mask, n)
        its = sim.step(u, w, 1)
        err = rel(u.cpu().numpy(), uo)
        assert err <= 1e-8, (n, err)
        assert abs(its[0] - res.iterations) <= 3
    sim.close()


def test_pcg_float32_reaches_tolerance_in_float64_residual():
    from paper_2602_16312_gb300 import aggmg
    wl = W.jittered_square_2d(n=30, n_levels=3)
    disc, ho = oracle_setup(wl)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f32")
    b = np.random.default_rng(22).standard_normal(disc.n)
    x = _dev(np.zeros(disc.n))
    res = hier.pcg_solve(_dev(b), x, rtol=1e-10, flexible=True)
    A0 = ho.levels[0].A
    r_true = np.linalg.norm(b - A0 @ x.cpu().numpy())
    assert r_true <= 1.01e-10 * np.linalg.norm(b)
    assert res["status"] == 0
