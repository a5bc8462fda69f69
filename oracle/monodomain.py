"""Monodomain time stepping: ionic models (Section 2.3) and the linearly
implicit step of Section 3.1 with ionic current interpolation.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per step (Section 3.1, the three bullet points after Eq. fully_discrete):
  1. ionic ODE at every DoF: w^{n+1} = w^n + dt H(u^n, w^n)
  2. ionic current at the DoFs, interpolated (ICI): the load is M f with
     f_i = I_app,i(t_{n+1}) - chi I_ion(U*_i, w_i^{n+1})
  3. solve A0 u^{n+1} = b by MG-PCG warm-started from u^n.

Schemes (mass coefficient c of A0 = c M + A):
  scheme 0, IMEX backward Euler (the workloads' form): c = chi C_m / dt,
      U* = u^n, w^{n+1} = w^n + dt H(u^n, w^n), b = M (c u^n + f).
  scheme 1, BDF2 with extrapolation (Eq. fully_discrete): c = 3 chi C_m / (2 dt),
      U* = 2u^n - u^{n-1}, W* = 2w^n - w^{n-1},
      w^{n+1} = (4 w^n - w^{n-1})/3 + (2 dt / 3) H(U*, W*)   (explicit BDF2),
      b = M (chi C_m (4 u^n - u^{n-1}) / (2 dt) + f), f with U* and w^{n+1}.
      Start (reading: the paper only asks for "suitable initializations"):
      u^{-1} = u^0 - dt u'(0), w^{-1} = w^0 - dt H(u^0, w^0), with u'(0) from
      the semi-discrete system, chi C_m u' = I_app - chi I_ion - M^{-1} A u;
      a first-order start would make the scheme first order.

Adjoint (not in the paper): the discrete adjoint of this recurrence. With
K = c M + A, a reverse step n+1 -> n takes ubar = dL/du^{n+1},
wbar = dL/dw^{n+1} and returns their values at step n and the per-element
log-conductivity gradient gamma_e = -lambda^T A_e u^{n+1} (A_e: part of A
built with D_e, see sipg.attributed_forms):
  lambda = K^{-1} ubar,  q = M lambda,
  wt = wbar - chi I_w(u^n, w^{n+1}) q,
  ubar_n = q (c - chi I_u(u^n, w^{n+1})) + dt H_u(u^n, w^n) wt,
  wbar_n = wt (1 + dt H_w(u^n, w^n)).
Pinned by central finite differences of the loss (tests).

Readings: the ionic ODE uses forward Euler (the workloads' "explicit
update"; the paper integrates it with BDF2). FitzHugh-Nagumo follows
Section 2.3.1 with k = 1, Gamma = b. Aliev-Panfilov is not in the paper; its
published form (Aliev & Panfilov 1996) is used:
  I_ion = k u (u - a)(u - 1) + u w,
  H     = (eps + mu1 w / (u + mu2)) (-w - k u (u - a - 1)).
Parity of these constants is unpinned by the paper (chosen readings); the
pins are the model equilibria and the space-clamped recurrence.
"""
from dataclasses import dataclass

import numpy as np

from .multigrid import pcg, vcycle

FHN, ALIEV_PANFILOV = 0, 1


def ionic(prm, u, w):
    """(I_ion(u, w), H(u, w)) of the model in prm (dict as in workloads)."""
    k, a, eps = prm["k"], prm["a"], prm["eps"]
    if prm["model"] == FHN:
        I = k * u * (u - a) * (u - 1.0) + w
        H = eps * (u - prm["gamma"] * w)
    else:
        mu1, mu2 = prm["mu1"], prm["mu2"]
        I = k * u * (u - a) * (u - 1.0) + u * w
        H = (eps + mu1 * w / (u + mu2)) * (-w - k * u * (u - a - 1.0))
    return I, H


def ionic_jacobian(prm, u, w):
    """Partial derivatives (I_u, I_w, H_u, H_w) of the model, pointwise."""
    k, a, eps = prm["k"], prm["a"], prm["eps"]
    dI_du = k * (3.0 * u * u - 2.0 * (a + 1.0) * u + a)
    if prm["model"] == FHN:
        g = prm["gamma"]
        return dI_du + 0.0 * w, np.ones_like(w), eps * np.ones_like(u), -eps * g * np.ones_like(w)
    mu1, mu2 = prm["mu1"], prm["mu2"]
    I_u = dI_du + w
    I_w = u.copy()
    e = eps + mu1 * w / (u + mu2)
    g = -w - k * u * (u - a - 1.0)
    e_u = -mu1 * w / (u + mu2) ** 2
    e_w = mu1 / (u + mu2)
    g_u = -k * (2.0 * u - a - 1.0)
    g_w = -1.0
    return I_u, I_w, e_u * g + e * g_u, e_w * g + e * g_w


@dataclass
class StepOptions:
    dt: float
    ionic: dict
    rtol: float = 1e-8
    max_it: int = 500
    chi: float = 1.0
    cm: float = 1.0
    iapp_value: float = 1.0
    iapp_steps: int = 5
    scheme: int = 0

    def mass_coeff(self):
        if self.scheme == 1:
            return 1.5 * self.chi * self.cm / self.dt
        return self.chi * self.cm / self.dt


def iapp(opts: StepOptions, mask, n):
    """Nodal applied current at t_{n+1}: iapp_value on the stimulated DoFs for
    the first iapp_steps steps (n = 0 .. iapp_steps-1), zero afterwards."""
    return opts.iapp_value * mask if n < opts.iapp_steps else np.zeros_like(mask)


def rhs(disc, opts: StepOptions, u, w_new, mask, n):
    """Load vector b of step n -> n+1 (ionic current interpolation: nodal f
    multiplied by the mass matrix)."""
    I, _ = ionic(opts.ionic, u, w_new)
    f = iapp(opts, mask, n) - opts.chi * I
    return disc.M @ (opts.mass_coeff() * u + f)


def step(disc, hier, opts: StepOptions, u, w, mask, n):
    """One backward-Euler time step n -> n+1. Returns (u_new, w_new, PCGResult)."""
    _, H = ionic(opts.ionic, u, w)
    w_new = w + opts.dt * H
    b = rhs(disc, opts, u, w_new, mask, n)
    A0 = hier.levels[0].A
    res = pcg(A0, b, u, lambda r: vcycle(hier, r), opts.rtol, opts.max_it)
    return res.x, w_new, res


def bdf2_start(disc, opts: StepOptions, u0, w0, mask):
    """History (u^{-1}, w^{-1}) of the BDF2 scheme from the state at t = 0."""
    import scipy.sparse.linalg as spl
    chi, cm, dt = opts.chi, opts.cm, opts.dt
    I, H = ionic(opts.ionic, u0, w0)
    f0 = iapp(opts, mask, 0) - chi * I
    MinvAu = spl.spsolve(disc.M.tocsc(), disc.A @ u0)
    udot = (f0 - MinvAu) / (chi * cm)
    return u0 - dt * udot, w0 - dt * H


def bdf2_step(disc, hier, opts: StepOptions, u, u_prev, w, w_prev, mask, n):
    """One BDF2 step n -> n+1 (scheme 1). Returns (u_new, w_new, PCGResult)."""
    chi, cm, dt = opts.chi, opts.cm, opts.dt
    ustar = 2.0 * u - u_prev
    wstar = 2.0 * w - w_prev
    _, H = ionic(opts.ionic, ustar, wstar)
    w_new = (4.0 * w - w_prev) / 3.0 + (2.0 * dt / 3.0) * H
    I, _ = ionic(opts.ionic, ustar, w_new)
    f = iapp(opts, mask, n) - chi * I
    b = disc.M @ (chi * cm / (2.0 * dt) * (4.0 * u - u_prev) + f)
    res = pcg(hier.levels[0].A, b, u, lambda r: vcycle(hier, r), opts.rtol, opts.max_it)
    return res.x, w_new, res


def run(disc, hier, opts: StepOptions, u0, w0, mask, n_steps):
    """n_steps time steps from (u0, w0); returns (u, w, iterations list)."""
    u, w = u0.copy(), w0.copy()
    its = []
    if opts.scheme == 1:
        u_prev, w_prev = bdf2_start(disc, opts, u0, w0, mask)
        for n in range(n_steps):
            u_new, w_new, res = bdf2_step(disc, hier, opts, u, u_prev, w, w_prev, mask, n)
            u_prev, w_prev, u, w = u, w, u_new, w_new
            its.append(res.iterations)
        return u, w, its
    for n in range(n_steps):
        u, w, res = step(disc, hier, opts, u, w, mask, n)
        its.append(res.iterations)
    return u, w, its


def adjoint_step(disc, hier, opts: StepOptions, forms, u_n, w_n, u_np1, ubar, wbar, rtol=1e-12):
    """Reverse of step(): returns (ubar_n, wbar_n, gamma)."""
    prm, dt, chi = opts.ionic, opts.dt, opts.chi
    c = opts.mass_coeff()
    _, H = ionic(prm, u_n, w_n)
    w_np1 = w_n + dt * H
    res = pcg(hier.levels[0].A, ubar, np.zeros_like(ubar), lambda r: vcycle(hier, r), rtol, 10 * opts.max_it)
    lam = res.x
    q = disc.M @ lam
    I_u, I_w, _, _ = ionic_jacobian(prm, u_n, w_np1)
    _, _, H_u, H_w = ionic_jacobian(prm, u_n, w_n)
    wt = wbar - chi * I_w * q
    ubar_n = q * (c - chi * I_u) + dt * H_u * wt
    wbar_n = wt * (1.0 + dt * H_w)
    from .sipg import attributed_bilinear
    gamma = -attributed_bilinear(forms, lam, u_np1, disc.B)
    return ubar_n, wbar_n, gamma


def trajectory(disc, hier, opts: StepOptions, u0, w0, mask, n_steps):
    """States u^0..u^N, w^0..w^N of run()."""
    us, ws = [u0.copy()], [w0.copy()]
    for n in range(n_steps):
        u, w, _ = step(disc, hier, opts, us[-1], ws[-1], mask, n)
        us.append(u)
        ws.append(w)
    return us, ws


def gradient_log_conductivity(disc, hier, opts: StepOptions, forms, us, ws, ubar_N, rtol=1e-12):
    """dL/d(log s_e) for a loss with dL/du^N = ubar_N (and no w^N term)."""
    ubar, wbar = ubar_N.copy(), np.zeros_like(ubar_N)
    gamma = np.zeros(disc.n_elements)
    for n in range(len(us) - 2, -1, -1):
        ubar, wbar, g = adjoint_step(disc, hier, opts, forms, us[n], ws[n], us[n + 1], ubar, wbar, rtol)
        gamma += g
    return gamma, ubar, wbar
