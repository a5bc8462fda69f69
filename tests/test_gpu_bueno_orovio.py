"""Bueno-Orovio model (Section 2.3.2, Eq. BuenoOrovio) on the GPU against the
oracle through the C ABI: the pointwise gate update, whole time steps of both
schemes with the three gates stored gate-major, and the cases it rejects."""
import dataclasses

import numpy as np
import pytest

from oracle import monodomain as omd
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
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _bo(wl):
    """The workload's mesh and levels with the Bueno-Orovio model, dt = 0.1 ms
    and a 500 /s stimulus for the first 1 ms."""
    return dataclasses.replace(wl, ionic=dict(W.BUENO_OROVIO), dt=1e-4, iapp_value=500.0, iapp_steps=10)


CASES = {
    "jcube3d_q2_6": lambda: _bo(W.jittered_cube_3d(n=6, degree=2, n_levels=3, group=2)),
    "shell_bo_q2": lambda: W.ventricle_shell_bo(16, 8, 4, n_levels=3),
    "jsquare2d_q2_30": lambda: _bo(W.jittered_square_2d(n=30, n_levels=3)),
}


def test_gate_update_matches_oracle():
    from paper_2602_16312_gb300 import aggmg
    p = W.BUENO_OROVIO
    rng = np.random.default_rng(21)
    n = 4099
    u = rng.uniform(-0.1, 1.6, n)
    w = rng.uniform(0.0, 1.0, (3, n))
    wd = _dev(w.reshape(-1))
    aggmg.ionic_update(p, 1e-4, _dev(u), wd)
    torch.cuda.synchronize()
    _, H = omd.ionic(p, u, w)
    assert rel(wd.cpu().numpy(), (w + 1e-4 * H).reshape(-1)) <= 1e-14
    with pytest.raises(ValueError):
        aggmg.ionic_update(p, 1e-4, _dev(u), _dev(w[0]))


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_trajectory_matches_oracle(name, scheme):
    from paper_2602_16312_gb300 import aggmg
    wl = CASES[name]()
    c = (1.5 if scheme == 1 else 1.0) / wl.dt
    disc, ho = oracle_setup(wl, c=c)
    opts = step_opts(wl)
    opts.scheme = scheme
    mask = wl.stim_mask_nodal()
    n_steps = 12
    w0 = np.repeat(W.resting_gates(wl.ionic)[:, None], disc.n, axis=1)
    u_ref, w_ref, its_ref = omd.run(disc, ho, opts, np.zeros(disc.n), w0, mask, n_steps)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), c, wl.maps, precision="f64")
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(mask), iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol, scheme=scheme)
    u = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    w = _dev(w0.reshape(-1))
    its = sim.step(u, w, 5) + sim.step(u, w, n_steps - 5)
    sim.close()
    assert its == its_ref
    assert rel(u.cpu().numpy(), u_ref) <= 1e-10
    assert rel(w.cpu().numpy(), w_ref.reshape(-1)) <= 1e-10
    # the stimulated tissue has crossed the excitation threshold V1
    assert u.max().item() > W.BUENO_OROVIO["V1"]


def test_rejections():
    from paper_2602_16312_gb300 import aggmg
    wl = CASES["jcube3d_q2_6"]()
    mesh = aggmg.Mesh.from_workload(wl, adjoint_data=True)
    hier = aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps, precision="f64")
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, rtol=wl.rtol)
    n = mesh.n_dofs
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):                       # one gate row where three are needed
        sim.step(u, torch.zeros(n, dtype=torch.float64, device="cuda"), 1)
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    grad = torch.zeros(mesh.n_elements, dtype=torch.float64, device="cuda")
    with pytest.raises(aggmg.AggError) as e:              # the adjoint covers one-gate models
        sim.adjoint_step(u, w, u, z.clone(), w.clone(), grad)
    assert e.value.status == aggmg.AGG_EUNSUPPORTED
    sim.close()
