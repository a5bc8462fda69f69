"""Pins of the oracle's adjoint (discrete adjoint of the time step; the paper
has no adjoint): attribution of A to elements, the log-conductivity
gradient against finite differences of the assembled operator, and the full
loss gradient against central differences of the forward run."""
import numpy as np
import pytest

from oracle import monodomain as omd
from oracle import multigrid as omg
from oracle import sipg
from paper_2602_16312_gb300 import workloads as W


def _setup(dim=2, n=3, p=2, jit=0.15):
    mesh = W.box_mesh(dim, n, jitter=jit, seed=9)
    if dim == 2:
        D = W.conductivity_from_fibres(W.planar_fibres(mesh.n_elements, 30.0), 1.2e-2, 2.5e-3)
    else:
        D = W.conductivity_from_fibres(W.rotating_fibres_z(mesh.centroids()), 1.2e-2, 2.5e-3)
    return mesh, D


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 1)])
def test_attributed_forms_sum_to_A_and_match_finite_differences(dim, p):
    mesh, D = _setup(dim=dim, n=3, p=p)
    disc = sipg.assemble(mesh.vertices, mesh.elements, D, p, 1, 10.0)
    forms = sipg.attributed_forms(mesh.vertices, mesh.elements, D, p, 1, 10.0)
    rng = np.random.default_rng(3)
    lam, u = rng.standard_normal(disc.n), rng.standard_normal(disc.n)
    g = sipg.attributed_bilinear(forms, lam, u, disc.B)
    assert abs(g.sum() - lam @ (disc.A @ u)) <= 1e-12 * np.abs(disc.A).max() * np.linalg.norm(lam) * np.linalg.norm(u)
    # dA/ds_e by central differences of the assembly with D_e scaled by (1 +- h)
    h = 1e-3
    for e in (0, mesh.n_elements // 2, mesh.n_elements - 1):
        Dp, Dm = D.copy(), D.copy()
        Dp[e] *= 1 + h
        Dm[e] *= 1 - h
        Ap = sipg.assemble(mesh.vertices, mesh.elements, Dp, p, 1, 10.0).A
        Am = sipg.assemble(mesh.vertices, mesh.elements, Dm, p, 1, 10.0).A
        fd = lam @ ((Ap - Am) @ u) / (2 * h)
        assert abs(g[e] - fd) <= 1e-9 * max(1.0, abs(fd))


def _loss_run(mesh, D0, theta, tmap, p, sensors, target, n_steps, opts):
    D = D0 * theta[tmap][:, None, None]
    disc = sipg.assemble(mesh.vertices, mesh.elements, D, p, 1, 10.0)
    hier = omg.build_hierarchy(disc, opts.mass_coeff(), [])      # direct solve: exact
    mask = np.repeat((np.arange(mesh.n_elements) < 3).astype(float), disc.B)
    us, ws = omd.trajectory(disc, hier, opts, np.zeros(disc.n), np.zeros(disc.n), mask, n_steps)
    elem, Wt = sensors
    val = np.einsum("si,si->s", Wt, us[-1].reshape(-1, disc.B)[elem])
    return float(np.sum((val - target) ** 2)), disc, hier, D, us, ws, val


@pytest.mark.parametrize("model", ["fhn", "ap"])
def test_theta_gradient_matches_central_differences(model):
    mesh, D0 = _setup(dim=2, n=4, p=1, jit=0.1)
    p = 1
    tmap, tshape = W.block_map(mesh.grid_shape, (2, 2))
    theta = np.exp(0.2 * np.random.default_rng(5).standard_normal(int(np.prod(tshape))))
    prm = dict(W.FHN, k=8.0, eps=0.05) if model == "fhn" else dict(W.ALIEV_PANFILOV, eps=0.02)
    opts = omd.StepOptions(dt=0.05, ionic=prm, rtol=1e-13, iapp_value=1.0, iapp_steps=3)
    pts = np.random.default_rng(6).uniform(0.05, 0.95, size=(9, 2))
    sensors = sipg.locate_points(mesh.vertices, mesh.elements, p, pts)
    n_steps = 6
    _, _, _, _, _, _, target = _loss_run(mesh, D0, np.ones_like(theta), tmap, p, sensors, 0.0, n_steps, opts)
    L, disc, hier, D, us, ws, val = _loss_run(mesh, D0, theta, tmap, p, sensors, target, n_steps, opts)
    elem, Wt = sensors
    ubar = np.zeros(disc.n)
    np.add.at(ubar.reshape(-1, disc.B), elem, 2 * (val - target)[:, None] * Wt)
    forms = sipg.attributed_forms(mesh.vertices, mesh.elements, D, p, 1, 10.0)
    gamma, _, _ = omd.gradient_log_conductivity(disc, hier, opts, forms, us, ws, ubar)
    grad = np.zeros_like(theta)
    np.add.at(grad, tmap, gamma)
    grad /= theta
    for k in range(len(theta)):
        h = 1e-5 * theta[k]
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        Lp = _loss_run(mesh, D0, tp, tmap, p, sensors, target, n_steps, opts)[0]
        Lm = _loss_run(mesh, D0, tm, tmap, p, sensors, target, n_steps, opts)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(grad[k] - fd) <= 1e-6 * max(np.abs(grad).max(), 1e-30), (k, grad[k], fd)


def test_locate_points_reproduces_polynomials():
    mesh, _ = _setup(dim=2, n=4, p=2, jit=0.2)
    pts = np.random.default_rng(8).uniform(0, 1, size=(20, 2))
    elem, Wt = sipg.locate_points(mesh.vertices, mesh.elements, 2, pts)
    xn = sipg.nodal_points(mesh.vertices, mesh.elements, 2)        # (E, B, 2)
    f = lambda x: 1 + 2 * x[..., 0] - x[..., 1] + 0.5 * x[..., 0] * x[..., 1]   # bilinear in physical space?
    # on a jittered (non-affine) mesh only affine functions are reproduced exactly
    g = lambda x: 1 + 2 * x[..., 0] - x[..., 1]
    vals = np.einsum("si,si->s", Wt, g(xn)[elem])
    np.testing.assert_allclose(vals, g(pts), atol=1e-12)
    del f


@pytest.mark.parametrize("model", ["fhn", "ap"])
def test_adjoint_step_is_the_transpose_of_the_step_linearisation(model):
    """Dot-product test of one reverse step: with J the Jacobian of the
    forward step (u^n, w^n) -> (u^{n+1}, w^{n+1}), taken here by central
    differences of the forward step, <J v, y> equals <v, J^T y> where
    J^T y = (ubar^n, wbar^n) is what adjoint_step returns for the seed y."""
    mesh, D = _setup(dim=2, n=3, p=2, jit=0.15)
    p = 2
    disc = sipg.assemble(mesh.vertices, mesh.elements, D, p, 1, 10.0)
    forms = sipg.attributed_forms(mesh.vertices, mesh.elements, D, p, 1, 10.0)
    prm = dict(W.FHN) if model == "fhn" else dict(W.ALIEV_PANFILOV)
    opts = omd.StepOptions(dt=0.05, ionic=prm, rtol=1e-14, iapp_value=1.0, iapp_steps=3)
    hier = omg.build_hierarchy(disc, opts.mass_coeff(), [])      # one level: the solves are direct
    rng = np.random.default_rng(12)
    n = disc.n
    u, w = rng.uniform(0.05, 0.9, n), rng.uniform(0.0, 0.3, n)
    du, dw = rng.standard_normal(n), rng.standard_normal(n)
    yu, yw = rng.standard_normal(n), rng.standard_normal(n)
    mask = np.repeat((np.arange(mesh.n_elements) < 2).astype(float), disc.B)
    h = 1e-5

    def forward(s):
        un, wn, _ = omd.step(disc, hier, opts, u + s * du, w + s * dw, mask, 0)
        return un, wn

    (up, wp), (um, wm) = forward(h), forward(-h)
    lhs = (up - um) @ yu / (2 * h) + (wp - wm) @ yw / (2 * h)
    u1, _ = forward(0.0)
    ubar_n, wbar_n, _ = omd.adjoint_step(disc, hier, opts, forms, u, w, u1, yu, yw, rtol=1e-14)
    rhs = du @ ubar_n + dw @ wbar_n
    scale = np.abs(du) @ np.abs(ubar_n) + np.abs(dw) @ np.abs(wbar_n)
    assert abs(lhs - rhs) <= 1e-8 * scale, (lhs, rhs)
