"""Shared helpers of the GPU parity tests (oracle side and device side)."""
import numpy as np

from oracle import monodomain as omd
from oracle import multigrid as omg
from oracle import sipg as osipg


def oracle_setup(wl, c=None):
    disc = osipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, wl.degree,
                          wl.penalty_mode, wl.penalty_coeff)
    c = 1.0 / wl.dt if c is None else c
    return disc, omg.build_hierarchy(disc, c, wl.maps)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def step_opts(wl, rtol=None):
    return omd.StepOptions(dt=wl.dt, ionic=wl.ionic, rtol=wl.rtol if rtol is None else rtol,
                           iapp_value=wl.iapp_value, iapp_steps=wl.iapp_steps)
