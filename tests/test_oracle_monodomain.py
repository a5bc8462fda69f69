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


# ---------------------------------------------------------------- Bueno-Orovio (Section 2.3.2)

def _bo_space_clamped(u0, t_end):
    """Space-clamped model u' = -I_ion(u, w), w' = H(u, w) from rest gates,
    integrated by an independent stiff solver (scipy LSODA, tight tolerances)."""
    from scipy.integrate import solve_ivp
    p = W.BUENO_OROVIO

    def f(t, y):
        I, H = md.ionic(p, y[:1], y[1:].reshape(3, 1))
        return np.concatenate([-I, H[:, 0]])

    y0 = np.concatenate([[u0], W.resting_gates(p)])
    return solve_ivp(f, (0.0, t_end), y0, method="LSODA", rtol=1e-9, atol=1e-11, max_step=1e-4,
                     dense_output=True)


def test_bueno_orovio_rest_is_equilibrium():
    p = W.BUENO_OROVIO
    w = W.resting_gates(p)[:, None]
    I, H = md.ionic(p, np.zeros(1), w)
    assert I[0] == 0.0 and np.all(H == 0.0)
    # the drift term as printed, (u - V_o), would leave a current -V_o / tau_o' at rest
    I2, _ = md.ionic(dict(p, uo=p["Vo"]), np.zeros(1), w)
    assert I2[0] == pytest.approx(-p["Vo"] / p["tauo_p"])


def test_bueno_orovio_gate_rates_above_thresholds():
    """Above V1 and V2 the a_i vanish: w0, w1 decay at 1/tau1+, 1/tau2+, and
    w2 relaxes to H^k3_V3(u) at 1/tau3''."""
    p = W.BUENO_OROVIO
    u = np.array([1.2, 1.5])
    w = np.array([[0.3, 0.7], [0.4, 0.9], [0.2, 0.5]])
    _, H = md.ionic(p, u, w)
    np.testing.assert_allclose(H[0], -w[0] / p["tau1plus"], rtol=1e-14)
    np.testing.assert_allclose(H[1], -w[1] / p["tau2plus"], rtol=1e-14)
    s_inf = 0.5 * (1.0 + np.tanh(p["k3"] * (u - p["V3"])))
    np.testing.assert_allclose(H[2], (s_inf - w[2]) / p["tau3pp"], rtol=1e-14)


def test_bueno_orovio_action_potential():
    """A supra-threshold start fires a full action potential: fast upstroke to
    near V^, a plateau of a few hundred ms, repolarisation to rest; a
    sub-threshold start (below V1) decays without an upstroke."""
    p = W.BUENO_OROVIO
    sol = _bo_space_clamped(0.5, 1.0)
    t = np.linspace(0.0, 1.0, 20001)
    u = sol.sol(t)[0]
    assert 1.3 < u.max() <= p["Vhat"]
    assert t[u.argmax()] < 2e-3
    above = t[u > 0.1 * u.max()]
    assert 0.15 < above.max() - above.min() < 0.45
    assert abs(u[-1]) < 0.05
    sub = _bo_space_clamped(0.2, 0.2)
    assert sub.y[0].max() <= 0.2 + 1e-12 and abs(sub.y[0, -1]) < 1e-3


def test_bueno_orovio_forward_euler_converges_to_space_clamped_solution():
    """The oracle's per-step order (gates by forward Euler, then the current
    with the new gates) converges at first order to the stiff solution."""
    p = W.BUENO_OROVIO
    ref = _bo_space_clamped(0.5, 0.05).sol(0.05)[0]
    errs = []
    for dt in (2e-5, 1e-5):
        u = np.array([0.5])
        w = W.resting_gates(p).reshape(3, 1).copy()
        for _ in range(int(round(0.05 / dt))):
            _, H = md.ionic(p, u, w)
            w = w + dt * H
            I, _ = md.ionic(p, u, w)
            u = u - dt * I
        errs.append(abs(u[0] - ref))
    assert errs[1] < 1e-2 and 1.6 < errs[0] / errs[1] < 2.4
