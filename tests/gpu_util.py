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
    """Element-wise error of a against the reference b: max_i |a_i - b_i|
    divided by max_i |b_i| (so one wrong entry among millions is not averaged
    away, as it would be in a 2-norm ratio)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    assert a.shape == b.shape, (a.shape, b.shape)
    return float(np.abs(a - b).max(initial=0.0) / max(np.abs(b).max(initial=0.0), 1e-300))


def worst(a, b):
    """Index, value and reference of the largest element-wise difference (for messages)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    i = int(np.argmax(np.abs(a - b)))
    return dict(index=i, got=float(a[i]), ref=float(b[i]), err=rel(a, b))


def step_opts(wl, rtol=None):
    return omd.StepOptions(dt=wl.dt, ionic=wl.ionic, rtol=wl.rtol if rtol is None else rtol,
                           iapp_value=wl.iapp_value, iapp_steps=wl.iapp_steps)
