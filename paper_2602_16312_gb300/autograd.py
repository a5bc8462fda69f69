"""Differentiable time stepping: a torch.autograd.Function around
agg_monodomain_step whose backward runs agg_monodomain_adjoint_step (the
discrete adjoint with the same MG-PCG) with checkpointing every K steps.

Parameters: per-block conductivity scales theta, D_e = theta[theta_map[e]] D0_e,
passed to the library with the mesh (agg_mesh_desc.theta / theta_map). The
reverse steps accumulate per-element log-conductivity gradients g_e on the
device, and agg_theta_gradient applies the chain rule dL/dtheta_k =
sum_{e: theta_map[e] = k} g_e / theta_k there. Only orchestration and
argument marshalling live here; every step, reverse step and reduction runs
in libaggmg.
"""
from __future__ import annotations

import numpy as np
import torch

from . import aggmg


class MonodomainProblem:
    """Geometry, reference conductivity D0, theta map and solver options of a
    differentiable simulation; `build(theta)` creates the library objects."""

    def __init__(self, wl, theta_map, precision="f64", rtol=1e-8, flexible=None, device="cuda"):
        self.wl = wl
        self.theta_map = np.asarray(theta_map, dtype=np.int64)
        self.precision = precision
        self.rtol = rtol
        self.flexible = (precision != "f64") if flexible is None else flexible
        self.device = torch.device(device)
        self.B = (wl.degree + 1) ** wl.mesh.dim
        self.n_dofs = wl.n_dofs
        self.mask = torch.tensor(wl.stim_mask_nodal(), dtype=torch.float64, device=self.device)
        self._built = None

    def build(self, theta: np.ndarray):
        mesh = aggmg.Mesh.from_workload(self.wl, adjoint_data=True, theta=np.asarray(theta, dtype=np.float64),
                                        theta_map=self.theta_map)
        hier = aggmg.Hierarchy(mesh, 1.0 / self.wl.dt, self.wl.maps, precision=self.precision)
        sim = aggmg.Monodomain(hier, self.wl.dt, self.wl.ionic, iapp_mask=self.mask, iapp_value=self.wl.iapp_value,
                               iapp_steps=self.wl.iapp_steps, rtol=self.rtol, flexible=self.flexible)
        self._built = (mesh, hier, sim)
        return self._built

    def sensors(self, points):
        """(elem, weights) tensors for point evaluation u_h(x_s) (library locate)."""
        mesh = self._built[0] if self._built else aggmg.Mesh.from_workload(self.wl)
        elem, w = mesh.locate(points)
        return (torch.tensor(elem, device=self.device), torch.tensor(w, dtype=torch.float64, device=self.device))

    def evaluate(self, u, sensors):
        elem, w = sensors
        return (u.view(-1, self.B)[elem] * w).sum(dim=1)


class MonodomainRun(torch.autograd.Function):
    """(u_N, w_N) = n_steps time steps from (u0, w0) with conductivity scales theta."""

    @staticmethod
    def forward(ctx, theta, u0, w0, problem: MonodomainProblem, n_steps: int, checkpoint_every: int = 20):
        mesh, hier, sim = problem.build(theta.detach().cpu().numpy())
        u, w = u0.detach().clone(), w0.detach().clone()
        sim.set_clock(0)
        ckpts = [(0, u.clone(), w.clone())]
        K = max(1, int(checkpoint_every))
        done = 0
        while done < n_steps:
            k = min(K, n_steps - done)
            sim.step(u, w, k, iters=False)
            done += k
            if done < n_steps:
                ckpts.append((done, u.clone(), w.clone()))
        ctx.problem = problem
        ctx.objs = (mesh, hier, sim)
        ctx.ckpts = ckpts
        ctx.n_steps = n_steps
        ctx.K = K
        ctx.save_for_backward(theta.detach())
        return u, w

    @staticmethod
    def backward(ctx, ubar_N, wbar_N):
        (theta,) = ctx.saved_tensors
        problem = ctx.problem
        _, _, sim = ctx.objs
        dev = problem.device
        N = problem.n_dofs
        ubar = ubar_N.detach().clone() if ubar_N is not None else torch.zeros(N, dtype=torch.float64, device=dev)
        wbar = wbar_N.detach().clone() if wbar_N is not None else torch.zeros(N, dtype=torch.float64, device=dev)
        ubar = ubar.contiguous()
        wbar = wbar.contiguous()
        grad = torch.zeros(problem.wl.mesh.n_elements, dtype=torch.float64, device=dev)
        for start, uc, wc in reversed(ctx.ckpts):
            end = min(start + ctx.K, ctx.n_steps)
            states = [(uc.clone(), wc.clone())]
            u, w = uc.clone(), wc.clone()
            sim.set_clock(start)
            for _ in range(start, end):
                sim.step(u, w, 1, iters=False)
                states.append((u.clone(), w.clone()))
            for n in range(end - 1, start - 1, -1):
                u_n, w_n = states[n - start]
                u_np1 = states[n - start + 1][0]
                sim.adjoint_step(u_n, w_n, u_np1, ubar, wbar, grad)
        _, hier, _ = ctx.objs
        gtheta = torch.zeros(theta.numel(), dtype=torch.float64, device=dev)
        hier.theta_gradient(grad, gtheta)
        return gtheta.to(theta.device), ubar, wbar, None, None, None
