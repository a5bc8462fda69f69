"""The CUDA path at the benchmark's full sizes, in the forms the workloads
name, against the oracle on every row:

  * the float64 operator A0 = c M + A (the outer CG's) and the V-cycle's
    level-0 operator applied to a seeded vector, element by element against
    the oracle's products (every block row, assembled chunk by chunk with the
    chunk's face neighbours, which gives each row exactly);
  * one time step from a seeded state: the gates at every DoF against the
    oracle's pointwise model, and the global true residual of the solve,
    ||b - A0 u^{n+1}|| with b = M (c u^n + I_app mask - I_ion(u^n, w^{n+1})),
    computed by the oracle on every row, within the solve's stopping
    criterion rtol ||b - A0 u^n||;
  * on the benchmark workload itself (512^2 Q2), the whole trajectory from
    rest through the stimulus steps against the oracle's own time steps,
    element by element: u and w after every step within 1e-8 of the oracle's
    largest entry in the float32 V-cycle form the benchmark times, and
    within 1e-10 with equal PCG iteration counts in the plain float64 form;
  * the V-cycle is symmetric and positive.
The oracle's products run in spawned worker processes (tests/oracle_rows.py);
the device hierarchy is released before they start."""
import gc
import os

import numpy as np
import pytest

import oracle_rows
from gpu_util import rel, worst
from oracle import monodomain as omd
from oracle import multigrid as omg
from oracle import sipg as osipg
from paper_2602_16312_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_16312_gb300 import build
    build.build()


CONFIGS = {
    # name: (workload, V-cycle form, V-cycle level-0 operator, chunks per grid axis, host GB per worker)
    "jsquare2d_q2_512_f32": ("W.jittered_square_2d(n=512, degree=2, n_levels=4)", "f32", "mf", (4, 4), 1.0),
    "jcube3d_q2_64_f32": ("W.jittered_cube_3d(n=64, degree=2, n_levels=4, group=4)", "f32", "mf", (4, 4, 4), 2.0),
    "jcube3d_q2_64_bf16s": ("W.jittered_cube_3d(n=64, degree=2, n_levels=4, group=4)", "bf16s", "mf", (4, 4, 4),
                            2.0),
    "shell_q2_128x96x16_f32": ("W.ventricle_shell()", "f32", "mf", (4, 4, 1), 3.0),
    "cube3d_q3_48_f64": ("W.cube_3d_adjoint(n=48)", "f64", "bsr", (4, 4, 4), 3.0),
    "cube3d_q3_48_f32": ("W.cube_3d_adjoint(n=48)", "f32", "mf", (4, 4, 4), 3.0),
}


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _workers(gb_each):
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) / 2**20
    except OSError:
        pass
    n = os.cpu_count() or 1
    if avail is not None:
        n = min(n, max(1, int(0.6 * avail / gb_each)))
    return max(1, min(n, 16))


@pytest.mark.parametrize("name", list(CONFIGS))
def test_full_size_every_row(name):
    from paper_2602_16312_gb300 import aggmg
    expr, form, fine, pieces, gb = CONFIGS[name]
    wl = eval(expr)
    N = wl.n_dofs
    c = 1.0 / wl.dt
    rng = np.random.default_rng(91)
    mesh = aggmg.Mesh.from_workload(wl)
    hier = aggmg.Hierarchy(mesh, c, wl.maps, precision=form, fine=fine, cheb_range=wl.cheb_range)

    # ---- the two level-0 operators on a seeded vector
    x = rng.standard_normal(N)
    y = torch.empty(N, dtype=torch.float64, device="cuda")
    hier.operator_apply(0, _dev(x), y)
    y_a0 = y.cpu().numpy()
    hier.operator_apply(-1, _dev(x), y)
    y_v0 = y.cpu().numpy()

    # ---- the V-cycle is symmetric and positive
    r1, r2 = _dev(rng.standard_normal(N)), _dev(rng.standard_normal(N))
    z1, z2 = torch.empty_like(r1), torch.empty_like(r2)
    hier.vcycle_apply(r1, z1)
    hier.vcycle_apply(r2, z2)
    a12, a21 = torch.dot(z1, r2).item(), torch.dot(z2, r1).item()
    sym_tol = 1e-12 if form == "f64" else 1e-4
    assert abs(a12 - a21) <= sym_tol * (abs(a12) + abs(a21))
    assert torch.dot(z1, r1).item() > 0 and torch.dot(z2, r2).item() > 0
    del r1, r2, z1, z2

    # ---- one time step from a seeded state
    u0 = rng.uniform(0.0, 0.3, N)
    ng = W.n_gates(wl.ionic)
    w0 = rng.uniform(0.0, 0.5, (ng, N)) if ng > 1 else rng.uniform(0.0, 0.5, N)
    mask = wl.stim_mask_nodal()
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(mask), iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol, flexible=(form != "f64"))
    u, w = _dev(u0), _dev(w0.ravel())
    its = sim.step(u, w, 1)
    u1, w1 = u.cpu().numpy(), w.cpu().numpy()
    sim.close()
    hier.close()
    mesh.close()
    del sim, hier, mesh, u, w, y
    gc.collect()
    torch.cuda.empty_cache()

    _, H = omd.ionic(wl.ionic, u0, w0)
    w_ref = w0 + wl.dt * H
    assert rel(w1, w_ref) <= 1e-13, worst(w1, w_ref)
    I, _ = omd.ionic(wl.ionic, u0, w_ref)
    vb = c * u0 + wl.iapp_value * mask - I

    # ---- the oracle's products on every row
    (Mx, Ax), (Mu0, Au0), (Mu1, Au1), (Mb, _) = oracle_rows.oracle_products(
        expr, wl.mesh.grid_shape, pieces, [x, u0, u1, vb], [(0, "MA"), (1, "MA"), (2, "MA"), (3, "M")],
        workers=_workers(gb))
    ref = c * Mx + Ax
    assert rel(y_a0, ref) <= 1e-12, worst(y_a0, ref)
    tol_v0 = 1e-12 if form == "f64" else 2e-6
    assert rel(y_v0, ref) <= tol_v0, worst(y_v0, ref)
    r0 = Mb - (c * Mu0 + Au0)
    r1 = Mb - (c * Mu1 + Au1)
    ratio = np.linalg.norm(r1) / np.linalg.norm(r0)
    print(f"{name}: {its} PCG iterations, true relative residual {ratio:.3e} (oracle, every row)")
    assert ratio <= 1.05 * wl.rtol, ratio


# ---------------------------------------------------------------- the benchmark's trajectory
TRAJ_STEPS = 6       # the 5 stimulus steps and the first step after them


@pytest.fixture(scope="module")
def bench_oracle_trajectory():
    """The oracle's time steps of the 512^2 Q2 workload from rest (u = w = 0)."""
    wl = W.jittered_square_2d(n=512, degree=2, n_levels=4)
    disc = osipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, wl.degree, wl.penalty_mode,
                          wl.penalty_coeff)
    ho = omg.build_hierarchy(disc, 1.0 / wl.dt, wl.maps, cheb_range=wl.cheb_range)
    opts = omd.StepOptions(dt=wl.dt, ionic=wl.ionic, rtol=wl.rtol, iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps)
    u, w = np.zeros(disc.n), np.zeros(disc.n)
    mask = wl.stim_mask_nodal()
    traj = []
    for k in range(TRAJ_STEPS):
        u, w, res = omd.step(disc, ho, opts, u, w, mask, k)
        traj.append((u.copy(), w.copy(), res.iterations))
    del disc, ho
    gc.collect()
    return wl, traj


@pytest.mark.parametrize("form", ["f32", "f64"])
def test_bench_workload_trajectory_matches_oracle(bench_oracle_trajectory, form):
    from paper_2602_16312_gb300 import aggmg
    wl, traj = bench_oracle_trajectory
    fine = "mf" if form == "f32" else "bsr"
    steps = TRAJ_STEPS if form == "f32" else 3
    mesh = aggmg.Mesh.from_workload(wl)
    hier = aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps, precision=form, fine=fine, cheb_range=wl.cheb_range)
    mask = _dev(wl.stim_mask_nodal())
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=mask, iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol, flexible=(form == "f32"))
    u = torch.zeros(wl.n_dofs, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(u)
    tol = 1e-8 if form == "f32" else 1e-10
    report = []
    for k in range(steps):
        its = sim.step(u, w, 1)
        uo, wo, ito = traj[k]
        eu, ew = rel(u.cpu().numpy(), uo), rel(w.cpu().numpy(), wo)
        report.append((k, its[0], ito, eu, ew))
        assert eu <= tol, (form, k, worst(u.cpu().numpy(), uo), report)
        assert ew <= tol, (form, k, worst(w.cpu().numpy(), wo), report)
        if form == "f64":
            assert its[0] == ito, (k, its, ito)
    print(f"{form}: step, iterations (GPU, oracle), max error u, w: {report}")
    sim.close()
    hier.close()
    mesh.close()
