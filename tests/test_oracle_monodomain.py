"""Pins of the oracle's ionic models and time stepping (Sections 2.3, 3.1)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import monodomain as md
from oracle import multigrid as mg
from oracle import sipg
from paper_2602_16312_gb300 import workloads as W


def test_model_equilibria():
    z = np.zeros(1)
    for prm in (W.FHN, W.ALIEV_PANFILOV):
        I, H = md.ionic(prm, z, z)
        assert I[0] == 0.0 and H[0] == 0.0
    # cubic roots of the Aliev-Panfilov current at w = 0
    u = np.array([0.0, W.ALIEV_PANFILOV["a"], 1.0])
    I, _ = md.ionic(W.ALIEV_PANFILOV, u, np.zeros(3))
    np.testing.assert_allclose(I, 0.0, atol=1e-16)
    # FHN: dw/dt = eps (u - Gamma w) vanishes on the line w = u / Gamma
    I, H = md.ionic(W.FHN, np.array([0.3]), np.array([0.3 / W.FHN["gamma"]]))
    assert abs(H[0]) < 1e-16


@pytest.mark.parametrize("prm", [W.FHN, W.ALIEV_PANFILOV])
def test_ionic_jacobian_matches_central_differences(prm):
    rng = np.random.default_rng(7)
    u = rng.uniform(-0.1, 1.1, 50)
    w = rng.uniform(0.0, 1.5, 50)
    h = 1e-6
    Iu, Iw, Hu, Hw = md.ionic_jacobian(prm, u, w)
    I_p, H_p = md.ionic(prm, u + h, w)
    I_m, H_m = md.ionic(prm, u - h, w)
    np.testing.assert_allclose(Iu, (I_p - I_m) / (2 * h), rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(Hu, (H_p - H_m) / (2 * h), rtol=1e-7, atol=1e-8)
    I_p, H_p = md.ionic(prm, u, w + h)
    I_m, H_m = md.ionic(prm, u, w - h)
    np.testing.assert_allclose(Iw, (I_p - I_m) / (2 * h), rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(Hw, (H_p - H_m) / (2 * h), rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("prm", [W.FHN, W.ALIEV_PANFILOV])
def test_space_clamped_dofs_follow_the_scalar_recurrence(prm):
    """Uniform state, no stimulus: A u = 0, so every DoF obeys
    u <- u - dt I(u, w_new), w_new = w + dt H(u, w) exactly."""
    wl = W.jittered_square_2d(n=8, n_levels=2)
    disc = sipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, 2, 1, 10.0)
    opts = md.StepOptions(dt=0.05, ionic=prm, rtol=1e-13)
    h = mg.build_hierarchy(disc, opts.mass_coeff(), wl.maps)
    u = np.full(disc.n, 0.35)
    w = np.full(disc.n, 0.02)
    mask = np.zeros(disc.n)
    u_s, w_s = 0.35, 0.02
    u_out, w_out, _ = md.run(disc, h, opts, u, w, mask, 6)
    for _ in range(6):
        _, Hs = md.ionic(prm, np.array([u_s]), np.array([w_s]))
        w_s = w_s + 0.05 * Hs[0]
        Is, _ = md.ionic(prm, np.array([u_s]), np.array([w_s]))
        u_s = u_s - 0.05 * Is[0]
    np.testing.assert_allclose(u_out, u_s, rtol=1e-11)
    np.testing.assert_allclose(w_out, w_s, rtol=1e-13)


@pytest.mark.parametrize("scheme,order", [(0, 1), (1, 2)])
def test_time_order_on_linear_diffusion(scheme, order):
    """Ionic current off (k = 0, eps = 0): u' = -M^{-1} A u is solved exactly by
    a matrix exponential; backward Euler converges at order 1, BDF2 with the
    derivative start at order 2."""
    mesh = W.box_mesh(2, 3, jitter=0.2, seed=8)
    D = W.isotropic_conductivity(mesh.n_elements, 2, 0.02)
    disc = sipg.assemble(mesh.vertices, mesh.elements, D, 1, 1, 10.0)
    prm = dict(W.FHN, k=0.0, eps=0.0)
    x = sipg.nodal_points(mesh.vertices, mesh.elements, 1).reshape(-1, 2)
    u0 = np.cos(np.pi * x[:, 0]) + 0.5 * x[:, 1] ** 2
    T = 0.4
    Md, Ad = disc.M.toarray(), disc.A.toarray()
    u_T = sla.expm(-np.linalg.solve(Md, Ad) * T) @ u0
    errs = []
    for nsteps in (8, 16, 32):
        dt = T / nsteps
        opts = md.StepOptions(dt=dt, ionic=prm, rtol=1e-13, iapp_steps=0, scheme=scheme)
        h = mg.build_hierarchy(disc, opts.mass_coeff(), [])
        u, _, _ = md.run(disc, h, opts, u0, np.zeros_like(u0), np.zeros_like(u0), nsteps)
        errs.append(np.linalg.norm(u - u_T))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > order - 0.15, (errs, rates)


@pytest.mark.parametrize("prm", [W.FHN, W.ALIEV_PANFILOV])
def test_bdf2_second_order_with_ionic_current(prm):
    """Self-convergence of the full BDF2 scheme (extrapolated ionic terms,
    explicit BDF2 gate update, derivative start) on the space-clamped ODE
    (uniform state: A u = 0): errors against a dt/16 run approach a 4x
    reduction per halving (asymptotic range)."""
    mesh = W.box_mesh(2, 2, jitter=0.1, seed=12)
    D = W.isotropic_conductivity(mesh.n_elements, 2, 0.01)
    disc = sipg.assemble(mesh.vertices, mesh.elements, D, 1, 1, 10.0)
    prm = dict(prm, k=2.0)
    u0 = np.full(disc.n, 0.4)
    w0 = np.full(disc.n, 0.05)
    T = 0.8

    def final(nsteps):
        opts = md.StepOptions(dt=T / nsteps, ionic=prm, rtol=1e-14, iapp_steps=0, scheme=1)
        h = mg.build_hierarchy(disc, opts.mass_coeff(), [])
        u, _, _ = md.run(disc, h, opts, u0, w0, np.zeros_like(u0), nsteps)
        return u[0]

    ref = final(2048)
    errs = [abs(final(n) - ref) for n in (32, 64, 128)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 1.85, (errs, rates)
