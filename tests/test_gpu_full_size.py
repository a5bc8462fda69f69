"""The CUDA path at the benchmark's full sizes, in the launch configuration
bench.py times (float32 V-cycle, the same level-0 operator), against the
oracle where it can compute outputs one by one, and by properties that hold
at any size:
  * sampled block rows of the float64 operator A0 = c M + A (the outer CG's)
    and of the V-cycle's level-0 operator: the oracle assembles each sampled
    element with its face neighbours, which gives that element's rows exactly;
  * one time step from a seeded state: the gate update at every DoF against
    the oracle's pointwise model; on the sampled elements, the solve's
    residual against the oracle's element-local right-hand side
    b_e = M_e (c u_e + I_app mask_e - I_ion(u_e, w_e^{n+1}));
  * PCG on A0 x = A0 x_true recovers x_true to its stopping criterion;
  * the V-cycle is symmetric and positive."""
import gc

import numpy as np
import pytest

from oracle import monodomain as omd
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
    # name: (workload, V-cycle form, level-0 operator), as bench.py runs them
    "jsquare2d_q2_512": (lambda: W.jittered_square_2d(n=512, degree=2, n_levels=4), "f32", "mf"),
    "jcube3d_q2_64": (lambda: W.jittered_cube_3d(n=64, degree=2, n_levels=4, group=4), "f32", "mf"),
    "shell_q2_128x96x16": (lambda: W.ventricle_shell(), "f32", "mf"),
    "cube3d_q3_48": (lambda: W.cube_3d_adjoint(n=48), "f32", "bsr"),
}


def _face_neighbours(elements, sample, dim):
    """Elements sharing a face (2^(d-1) vertices) with each sampled element."""
    nv = 1 << (dim - 1)
    flat = elements.ravel()
    order = np.argsort(flat, kind="stable")
    starts = np.searchsorted(flat[order], np.arange(flat.max() + 2))
    out = set(int(e) for e in sample)
    for e in sample:
        cand = np.concatenate([order[starts[v]:starts[v + 1]] // elements.shape[1] for v in elements[e]])
        ids, counts = np.unique(cand, return_counts=True)
        out.update(int(i) for i in ids[(counts >= nv) & (ids != e)])
    return np.array(sorted(out), dtype=np.int64)


def _rows(disc, idx, x, local, B):
    """Block rows of the sampled elements of (M, A) applied to x (global)."""
    xs = x.reshape(-1, B)[idx].ravel()
    r = np.concatenate([np.arange(local[e] * B, local[e] * B + B) for e in local])
    return disc.M[r] @ xs, disc.A[r] @ xs


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name", list(CONFIGS))
def test_full_size(name):
    from paper_2602_16312_gb300 import aggmg
    make, form, fine = CONFIGS[name]
    wl = make()
    B, E, N = (wl.degree + 1) ** wl.mesh.dim, wl.mesh.n_elements, wl.n_dofs
    c = 1.0 / wl.dt
    mesh = aggmg.Mesh.from_workload(wl)
    hier = aggmg.Hierarchy(mesh, c, wl.maps, precision=form, fine=fine)
    rng = np.random.default_rng(91)
    # sampled elements: seeded random ones plus the first and last element
    sample = np.unique(np.concatenate([rng.choice(E, 48, replace=False), [0, E - 1]]))
    idx = _face_neighbours(wl.mesh.elements, sample, wl.mesh.dim)
    disc = osipg.assemble(wl.mesh.vertices, wl.mesh.elements[idx], wl.conductivity[idx], wl.degree,
                          wl.penalty_mode, wl.penalty_coeff)
    local = {int(e): int(np.searchsorted(idx, e)) for e in sample}
    rows = np.concatenate([np.arange(e * B, e * B + B) for e in sample])

    # ---- sampled rows of the float64 operator and of the V-cycle's level-0 operator
    x = rng.standard_normal(N)
    Mx, Ax = _rows(disc, idx, x, local, B)
    ref = c * Mx + Ax
    y = torch.empty(N, dtype=torch.float64, device="cuda")
    hier.operator_apply(0, _dev(x), y)
    got = y.cpu().numpy()[rows]
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    hier.operator_apply(-1, _dev(x), y)
    got = y.cpu().numpy()[rows]
    assert np.linalg.norm(got - ref) <= 2e-6 * np.linalg.norm(ref)

    # ---- one time step from a seeded state
    u0 = rng.uniform(0.0, 0.3, N)
    ng = W.n_gates(wl.ionic)
    w0 = rng.uniform(0.0, 0.5, (ng, N)) if ng > 1 else rng.uniform(0.0, 0.5, N)
    mask = wl.stim_mask_nodal()
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(mask), iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol, flexible=(form != "f64"))
    u, w = _dev(u0), _dev(w0.ravel())
    sim.step(u, w, 1)
    sim.close()
    _, H = omd.ionic(wl.ionic, u0, w0)
    w_ref = w0 + wl.dt * H
    assert np.abs(w.cpu().numpy() - w_ref.ravel()).max() <= 1e-13 * max(1.0, np.abs(w_ref).max())
    I, _ = omd.ionic(wl.ionic, u0, w_ref)
    f = wl.iapp_value * mask - I
    Mb, _ = _rows(disc, idx, c * u0 + f, local, B)
    u1 = u.cpu().numpy()
    Mu, Au = _rows(disc, idx, u1, local, B)
    r_s = Mb - (c * Mu + Au)
    assert np.linalg.norm(r_s) <= 1e-5 * np.linalg.norm(Mb)

    # ---- PCG on A0 x = A0 x_true
    x_true = _dev(rng.standard_normal(N))
    b = torch.empty_like(x_true)
    hier.operator_apply(0, x_true, b)
    xs = torch.zeros_like(x_true)
    res = hier.pcg_solve(b, xs, rtol=1e-8, flexible=(form != "f64"))
    r = torch.empty_like(b)
    hier.operator_apply(0, xs, r)
    assert (torch.linalg.norm(b - r) / torch.linalg.norm(b)).item() <= 1.05e-8
    assert res["iterations"] < 200

    # ---- the V-cycle is symmetric and positive
    r1, r2 = _dev(rng.standard_normal(N)), _dev(rng.standard_normal(N))
    z1, z2 = torch.empty_like(r1), torch.empty_like(r2)
    hier.vcycle_apply(r1, z1)
    hier.vcycle_apply(r2, z2)
    a12, a21 = torch.dot(z1, r2).item(), torch.dot(z2, r1).item()
    assert abs(a12 - a21) <= 1e-4 * (abs(a12) + abs(a21))
    assert torch.dot(z1, r1).item() > 0 and torch.dot(z2, r2).item() > 0
    hier.close()
    mesh.close()
    del hier, mesh
    gc.collect()
