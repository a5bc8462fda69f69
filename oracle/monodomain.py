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

Bueno-Orovio (Section 2.3.2, Eq. BuenoOrovio; model 2): three gates
w = (w0, w1, w2), each dw_i/dt = (b_i - a_i) w_i + a_i w_i^inf, with
H_z0(z) the unit step at z0 (1 for z >= z0) and H^k_z0(z) = (1 + tanh(k (z - z0)))/2:
  a0 = (1 - H_V1) / (H_V1m (tau1'' - tau1') + tau1'),   b0 = -H_V1 / tau1+,
  w0^inf = 1 - H_V1m,
  a1 = (1 - H_V2) / (H^k2_V2m (tau2'' - tau2') + tau2'), b1 = -H_V2 / tau2+,
  w1^inf = H_Vo (w*inf - 1 + u / tau2inf) + 1 - u / tau2inf,
  a2 = 1 / (H_V2 (tau3'' - tau3') + tau3'),              b2 = 0,
  w2^inf = H^k3_V3,
  I_ion = I_fi + I_so + I_si,
  I_fi = -H_V1 (u - V1)(Vhat - u) w0 / tau_fi,
  I_so = (1 - H_V2)(u - uo) / (H_Vo (tau_o'' - tau_o') + tau_o')
         + H_V2 / (H^kso_Vso (tau_so'' - tau_so') + tau_so'),
  I_si = -H_V2 w1 w2 / tau_si.
Readings: the superscript "-" of H in a0 and w0^inf is the threshold V1m
(V1^- in the text), the one of H in a1 is the smoothed step at V2m with
slope k2; w2^inf uses V3 with slope k3; the paper prints (u - V_o) in I_so,
but with it the resting state u = 0, w = (1, 1, H^k3_V3(0)) carries the
current -V_o / tau_o' = -1 and is not an equilibrium, so the model's
reference potential uo = 0 is used (tests pin the equilibrium). Parameter
values: the appendix table with its repeated rows taken once. The adjoint
is built for models 0 and 1 only.
"""
from dataclasses import dataclass

import numpy as np

from .multigrid import pcg, vcycle

FHN, ALIEV_PANFILOV, BUENO_OROVIO = 0, 1, 2


def _step(z, z0):
    """Unit step at z0: 1 where z >= z0."""
    return (np.asarray(z) >= z0).astype(float)


def _smooth_step(z, z0, k):
    return 0.5 * (1.0 + np.tanh(k * (np.asarray(z) - z0)))


def bueno_orovio(p, u, w):
    """(I_ion, H) of the Bueno-Orovio model; w has one row per gate (3, n)."""
    w0, w1, w2 = w[0], w[1], w[2]
    H_V1, H_V1m = _step(u, p["V1"]), _step(u, p["V1m"])
    H_V2, H_Vo = _step(u, p["V2"]), _step(u, p["Vo"])
    a0 = (1.0 - H_V1) / (H_V1m * (p["tau1pp"] - p["tau1p"]) + p["tau1p"])
    b0 = -H_V1 / p["tau1plus"]
    w0_inf = 1.0 - H_V1m
    a1 = (1.0 - H_V2) / (_smooth_step(u, p["V2m"], p["k2"]) * (p["tau2pp"] - p["tau2p"]) + p["tau2p"])
    b1 = -H_V2 / p["tau2plus"]
    w1_inf = H_Vo * (p["winf_star"] - 1.0 + u / p["tau2inf"]) + 1.0 - u / p["tau2inf"]
    a2 = 1.0 / (H_V2 * (p["tau3pp"] - p["tau3p"]) + p["tau3p"])
    w2_inf = _smooth_step(u, p["V3"], p["k3"])
    H = np.stack([(b0 - a0) * w0 + a0 * w0_inf,
                  (b1 - a1) * w1 + a1 * w1_inf,
                  -a2 * w2 + a2 * w2_inf])
    I_fi = -H_V1 * (u - p["V1"]) * (p["Vhat"] - u) * w0 / p["taufi"]
    I_so = ((1.0 - H_V2) * (u - p["uo"]) / (H_Vo * (p["tauo_pp"] - p["tauo_p"]) + p["tauo_p"])
            + H_V2 / (_smooth_step(u, p["Vso"], p["kso"]) * (p["tauso_pp"] - p["tauso_p"]) + p["tauso_p"]))
    I_si = -H_V2 * w1 * w2 / p["tausi"]
    return I_fi + I_so + I_si, H


def ionic(prm, u, w):
    """(I_ion(u, w), H(u, w)) of the model in prm (dict as in workloads).
    Models 0, 1: w and H have the shape of u; model 2: one row per gate."""
    if prm["model"] == BUENO_OROVIO:
        return bueno_orovio(prm, u, w)
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
    """Partial derivatives (I_u, I_w, H_u, H_w) of the model, pointwise
    (models 0 and 1)."""
    if prm["model"] == BUENO_OROVIO:
        raise NotImplementedError("the adjoint is built for the one-gate models")
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
