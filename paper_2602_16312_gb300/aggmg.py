"""ctypes binding of libaggmg (include/aggmg.h): argument marshalling only.

Every computation runs in the library; this module converts numpy arrays
(host inputs) and torch tensors (device vectors, via data_ptr()) to the C
ABI, and raises AggError on a non-zero status. The library must have been
built (`paper_2602_16312_gb300.build.build()`); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

AGG_OK, AGG_EINVAL, AGG_ENOMEM, AGG_ECUDA, AGG_ENOTSPD, AGG_ENOTCONV, AGG_ENAN, AGG_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7)
AGG_F64, AGG_F32, AGG_F32_BF16SMOOTH = 0, 1, 2
PRECISIONS = {"f64": AGG_F64, "f32": AGG_F32, "bf16s": AGG_F32_BF16SMOOTH}
AGG_FHN, AGG_ALIEV_PANFILOV, AGG_BUENO_OROVIO = 0, 1, 2


class AggError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("degree", C.c_int), ("n_vertices", C.c_int64), ("n_elements", C.c_int64),
                ("vertices", C.POINTER(C.c_double)), ("elements", C.POINTER(C.c_int64)),
                ("conductivity", C.POINTER(C.c_double)), ("penalty_mode", C.c_int),
                ("penalty_coeff", C.c_double), ("quad_extra", C.c_int), ("adjoint_data", C.c_int),
                ("theta", C.POINTER(C.c_double)), ("theta_map", C.POINTER(C.c_int32)), ("n_theta", C.c_int64)]


class MGOpts(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("agg_maps", C.POINTER(C.POINTER(C.c_int32))),
                ("smoother_degree", C.c_int), ("block_jacobi", C.c_int), ("lanczos_steps", C.c_int),
                ("cheb_upper_safety", C.c_double), ("cheb_range", C.c_double), ("vcycle_precision", C.c_int),
                ("fine_operator", C.c_int), ("coarse_persistent", C.c_int), ("coarse_cluster", C.c_int),
                ("coarse_operator", C.c_int)]


class PCGOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("max_it", C.c_int), ("flexible", C.c_int)]


class PCGResult(C.Structure):
    _fields_ = [("iterations", C.c_int), ("r0_norm", C.c_double), ("r_norm", C.c_double), ("status", C.c_int)]


BO_FIELDS = ("tau1p", "tau1pp", "tau1plus", "tau2p", "tau2pp", "tau2plus", "tau2inf", "tau3p", "tau3pp",
             "taufi", "tauo_p", "tauo_pp", "tauso_p", "tauso_pp", "tausi", "k2", "k3", "kso", "winf_star",
             "V1", "V1m", "V2", "V2m", "V3", "Vhat", "Vo", "Vso", "uo")


class BuenoOrovioParams(C.Structure):
    _fields_ = [(f, C.c_double) for f in BO_FIELDS]


class IonicParams(C.Structure):
    _fields_ = [("model", C.c_int), ("k", C.c_double), ("a", C.c_double), ("eps", C.c_double),
                ("gamma", C.c_double), ("mu1", C.c_double), ("mu2", C.c_double), ("bo", BuenoOrovioParams)]


class SimOpts(C.Structure):
    _fields_ = [("dt", C.c_double), ("chi_m", C.c_double), ("c_m", C.c_double), ("ionic", IonicParams),
                ("iapp_mask_dev", C.c_void_p), ("iapp_value", C.c_double), ("iapp_steps", C.c_int),
                ("pcg", PCGOpts), ("scheme", C.c_int)]


_lib = None

_SIGS = {
    "agg_dg_mesh_create": [C.POINTER(MeshDesc), C.POINTER(C.c_void_p)],
    "agg_dg_mesh_destroy": [C.c_void_p],
    "agg_dg_mesh_info": [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "agg_dg_mesh_nnzb": [C.c_void_p, C.POINTER(C.c_int64)],
    "agg_dg_mesh_locate": [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
    "agg_monodomain_adjoint_step": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p],
    "agg_dg_mesh_copy": [C.c_void_p, C.c_int, C.c_void_p],
    "agg_mg_opts_default": [C.POINTER(MGOpts)],
    "agg_mg_hierarchy_setup": [C.c_void_p, C.c_double, C.POINTER(MGOpts), C.c_void_p, C.POINTER(C.c_void_p)],
    "agg_mg_hierarchy_destroy": [C.c_void_p],
    "agg_hier_stats": [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                       C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "agg_pcg_solve": [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(PCGOpts), C.POINTER(PCGResult), C.c_void_p],
    "agg_operator_apply": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
    "agg_vcycle_apply": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "agg_operator_apply_static": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
    "agg_ionic_update": [C.POINTER(IonicParams), C.c_double, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
    "agg_rtree_agglomerate": [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.POINTER(C.c_int32)),
                              C.POINTER(C.c_int64), C.POINTER(C.c_int)],
    "agg_monodomain_create": [C.c_void_p, C.POINTER(SimOpts), C.POINTER(C.c_void_p)],
    "agg_monodomain_step": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.c_void_p],
    "agg_monodomain_set_clock": [C.c_void_p, C.c_int64],
    "agg_monodomain_destroy": [C.c_void_p],
    "agg_host_hierarchy_build": [C.c_void_p, C.c_double, C.POINTER(MGOpts), C.POINTER(C.c_void_p)],
    "agg_host_hierarchy_destroy": [C.c_void_p],
    "agg_host_hierarchy_level": [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_double)],
    "agg_host_hierarchy_copy": [C.c_void_p, C.c_int, C.c_int, C.c_void_p],
    "agg_profile_kernel": [C.c_void_p, C.c_int, C.c_int, C.c_void_p],
    "agg_kernel_cost": [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "agg_theta_gradient": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "agg_hier_launches": [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                          C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "agg_status_string": [C.c_int],
    "agg_last_error": [],
}


def lib():
    """Loads libaggmg.so from the package's build folder (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libaggmg.so is not built ({path}); run paper_2602_16312_gb300.build.build()")
    L = C.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.agg_status_string.restype = C.c_char_p
    L.agg_last_error.restype = C.c_char_p
    L.agg_mg_opts_default.restype = None
    _lib = L
    return L


def exported_symbols() -> List[str]:
    return list(_SIGS)


def _check(status):
    if status != AGG_OK:
        msg = lib().agg_last_error().decode(errors="replace")
        raise AggError(status, msg or lib().agg_status_string(status).decode())


def _dptr(t) -> int:
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 tensor")
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


# ---------------------------------------------------------------- mesh
class Mesh:
    """agg_dg_mesh_create: SIPG stiffness and element mass blocks (host FP64)."""

    def __init__(self, vertices, elements, conductivity, degree, penalty_mode=1, penalty_coeff=10.0,
                 quad_extra=1, adjoint_data=False, theta=None, theta_map=None):
        self.vertices = np.ascontiguousarray(vertices, dtype=np.float64)
        self.elements = np.ascontiguousarray(elements, dtype=np.int64)
        self.conductivity = np.ascontiguousarray(conductivity, dtype=np.float64)
        self.dim = self.vertices.shape[1]
        self.degree = degree
        self.B = (degree + 1) ** self.dim
        self.n_elements = self.elements.shape[0]
        th, tm, nth = None, None, 0
        if theta is not None:
            self.theta = np.ascontiguousarray(theta, dtype=np.float64)
            self.theta_map = np.ascontiguousarray(theta_map, dtype=np.int32)
            th = self.theta.ctypes.data_as(C.POINTER(C.c_double))
            tm = self.theta_map.ctypes.data_as(C.POINTER(C.c_int32))
            nth = len(self.theta)
        d = MeshDesc(self.dim, degree, self.vertices.shape[0], self.n_elements,
                     self.vertices.ctypes.data_as(C.POINTER(C.c_double)),
                     self.elements.ctypes.data_as(C.POINTER(C.c_int64)),
                     self.conductivity.ctypes.data_as(C.POINTER(C.c_double)),
                     penalty_mode, penalty_coeff, quad_extra, int(adjoint_data), th, tm, nth)
        h = C.c_void_p()
        _check(lib().agg_dg_mesh_create(C.byref(d), C.byref(h)))
        self.handle = h

    @classmethod
    def from_workload(cls, wl, conductivity=None, adjoint_data=False, theta=None, theta_map=None):
        D = wl.conductivity if conductivity is None else conductivity
        return cls(wl.mesh.vertices, wl.mesh.elements, D, wl.degree, wl.penalty_mode, wl.penalty_coeff,
                   adjoint_data=adjoint_data, theta=theta, theta_map=theta_map)

    def locate(self, points):
        """(elem, weights) of agg_dg_mesh_locate for host points (n, dim)."""
        pts = np.ascontiguousarray(points, dtype=np.float64)
        elem = np.empty(len(pts), np.int64)
        w = np.empty((len(pts), self.B), np.float64)
        _check(lib().agg_dg_mesh_locate(self.handle, len(pts), pts.ctypes.data, elem.ctypes.data, w.ctypes.data))
        return elem, w

    @property
    def n_dofs(self):
        return self.n_elements * self.B

    def info(self):
        nd, nf = C.c_int64(), C.c_int64()
        _check(lib().agg_dg_mesh_info(self.handle, C.byref(nd), C.byref(nf)))
        return nd.value, nf.value

    def stiffness_bsr(self):
        """(rowptr, cols, blocks) of the SIPG stiffness in element order."""
        nnzb = C.c_int64()
        _check(lib().agg_dg_mesh_nnzb(self.handle, C.byref(nnzb)))
        rp = np.empty(self.n_elements + 1, np.int64)
        cols = np.empty(nnzb.value, np.int32)
        vals = np.empty((nnzb.value, self.B, self.B), np.float64)
        for what, arr in ((0, rp), (1, cols), (2, vals)):
            _check(lib().agg_dg_mesh_copy(self.handle, what, arr.ctypes.data))
        return rp, cols, vals

    def element_mass(self):
        out = np.empty((self.n_elements, self.B, self.B))
        _check(lib().agg_dg_mesh_copy(self.handle, 3, out.ctypes.data))
        return out

    def adjoint_forms(self):
        """(Ke (E,B,B), Y (nnzb,4,B,B)) of a mesh made with adjoint_data."""
        nnzb = C.c_int64()
        _check(lib().agg_dg_mesh_nnzb(self.handle, C.byref(nnzb)))
        Ke = np.empty((self.n_elements, self.B, self.B))
        Y = np.empty((nnzb.value, 4, self.B, self.B))
        _check(lib().agg_dg_mesh_copy(self.handle, 5, Ke.ctypes.data))
        _check(lib().agg_dg_mesh_copy(self.handle, 6, Y.ctypes.data))
        return Ke, Y

    def volumes(self):
        out = np.empty(self.n_elements)
        _check(lib().agg_dg_mesh_copy(self.handle, 4, out.ctypes.data))
        return out

    def close(self):
        if self.handle:
            lib().agg_dg_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


FINE_OPERATORS = {"bsr": 0, "mf": 1}


def _mg_opts(maps: Sequence[np.ndarray], precision="f64", block_jacobi=True, lanczos_steps=12,
             safety=1.2, cheb_range=20.0, fine="bsr", coarse_persistent=False, coarse_cluster=False,
             coarse_operator="inherited"):
    o = MGOpts()
    lib().agg_mg_opts_default(C.byref(o))
    keep = [np.ascontiguousarray(m, dtype=np.int32) for m in maps]
    arr = (C.POINTER(C.c_int32) * max(1, len(keep)))()
    for i, m in enumerate(keep):
        arr[i] = m.ctypes.data_as(C.POINTER(C.c_int32))
    o.n_levels = len(keep) + 1
    o.agg_maps = C.cast(arr, C.POINTER(C.POINTER(C.c_int32)))
    o.block_jacobi = int(block_jacobi)
    o.lanczos_steps = lanczos_steps
    o.cheb_upper_safety = safety
    o.cheb_range = cheb_range
    o.vcycle_precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.fine_operator = FINE_OPERATORS[fine] if isinstance(fine, str) else int(fine)
    o.coarse_persistent = int(coarse_persistent)
    o.coarse_cluster = int(coarse_cluster)
    o.coarse_operator = {"inherited": 0, "direct": 1}[coarse_operator] if isinstance(coarse_operator, str) \
        else int(coarse_operator)
    return o, (keep, arr)


class HostHierarchy:
    """agg_host_hierarchy_build: the float64 set-up without a device."""

    def __init__(self, mesh: Mesh, mass_coeff: float, maps, **kw):
        o, self._keep = _mg_opts(maps, **kw)
        h = C.c_void_p()
        _check(lib().agg_host_hierarchy_build(mesh.handle, mass_coeff, C.byref(o), C.byref(h)))
        self.handle = h
        self.B = mesh.B
        self.n_levels = o.n_levels

    def level(self, l):
        n, nnzb, lam = C.c_int64(), C.c_int64(), C.c_double()
        _check(lib().agg_host_hierarchy_level(self.handle, l, C.byref(n), C.byref(nnzb), C.byref(lam)))
        return n.value, nnzb.value, lam.value

    def copy(self, l, what):
        n, nnzb, _ = self.level(l)
        B = self.B
        spec = {0: (np.int64, (n,)), 1: (np.int64, (n + 1,)), 2: (np.int32, (nnzb,)),
                3: (np.float64, (nnzb, B, B)), 4: (np.float64, (n, B, B)), 5: (np.float64, (n, B, B)),
                6: (np.int32, (n,))}[what]
        out = np.empty(spec[1], spec[0])
        _check(lib().agg_host_hierarchy_copy(self.handle, l, what, out.ctypes.data))
        return out

    def close(self):
        if self.handle:
            lib().agg_host_hierarchy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """agg_mg_hierarchy_setup: host set-up + upload + CUDA graphs."""

    def __init__(self, mesh: Mesh, mass_coeff: float, maps, precision="f64", stream=None, **kw):
        o, self._keep = _mg_opts(maps, precision=precision, **kw)
        h = C.c_void_p()
        _check(lib().agg_mg_hierarchy_setup(mesh.handle, mass_coeff, C.byref(o), C.c_void_p(_stream(stream)),
                                            C.byref(h)))
        self.handle = h
        self.mesh = mesh
        self.n_levels = o.n_levels
        self.mass_coeff = mass_coeff

    def stats(self):
        L = self.n_levels
        units = (C.c_int64 * L)()
        nnzb = (C.c_int64 * L)()
        lam = (C.c_double * L)()
        oc = C.c_double()
        nl = C.c_int()
        _check(lib().agg_hier_stats(self.handle, C.byref(nl), units, nnzb, lam, C.byref(oc)))
        return dict(units=list(units), nnzb=list(nnzb), lambda_max=list(lam)[:L - 1], op_complexity=oc.value)

    def pcg_solve(self, b, x, rtol=1e-8, atol=0.0, max_it=500, flexible=False, stream=None, check=True):
        o = PCGOpts(rtol, atol, max_it, int(flexible))
        r = PCGResult()
        st = lib().agg_pcg_solve(self.handle, C.c_void_p(_dptr(b)), C.c_void_p(_dptr(x)), C.byref(o),
                                 C.byref(r), C.c_void_p(_stream(stream)))
        if check and st not in (AGG_OK,):
            _check(st)
        return dict(iterations=r.iterations, r0_norm=r.r0_norm, r_norm=r.r_norm, status=r.status)

    def operator_apply(self, level, x, y, stream=None):
        _check(lib().agg_operator_apply(self.handle, level, C.c_void_p(_dptr(x)), C.c_void_p(_dptr(y)),
                                        C.c_void_p(_stream(stream))))

    def operator_apply_static(self, level, x, y, stream=None):
        """agg_operator_apply_static: same product, scratch in the library's
        static device array (no allocation during the call)."""
        _check(lib().agg_operator_apply_static(self.handle, level, C.c_void_p(_dptr(x)), C.c_void_p(_dptr(y)),
                                               C.c_void_p(_stream(stream))))

    def vcycle_apply(self, r, z, stream=None):
        _check(lib().agg_vcycle_apply(self.handle, C.c_void_p(_dptr(r)), C.c_void_p(_dptr(z)),
                                      C.c_void_p(_stream(stream))))

    def profile_kernel(self, kernel, reps, stream=None):
        _check(lib().agg_profile_kernel(self.handle, kernel, reps, C.c_void_p(_stream(stream))))

    def theta_gradient(self, grad_logD, theta_grad, stream=None):
        """agg_theta_gradient: theta_grad[k] += sum_{e in k} grad_logD[e] / theta[k]
        (device tensors; the mesh's conductivity parameters)."""
        _check(lib().agg_theta_gradient(self.handle, C.c_void_p(_dptr(grad_logD)), C.c_void_p(_dptr(theta_grad)),
                                        C.c_void_p(_stream(stream))))

    def launches(self):
        """agg_hier_launches: kernel launches per V-cycle, per PCG iteration and
        per solve set-up, and whether the coarse levels run persistently."""
        v, i, s, p, cl, cc = (C.c_int() for _ in range(6))
        _check(lib().agg_hier_launches(self.handle, C.byref(v), C.byref(i), C.byref(s), C.byref(p), C.byref(cl),
                                       C.byref(cc)))
        return dict(per_vcycle=v.value, per_iteration=i.value, per_setup=s.value, persistent=bool(p.value),
                    cluster_level=cl.value, cluster_ctas=cc.value)

    def kernel_cost(self, kernel):
        b, f = C.c_double(), C.c_double()
        _check(lib().agg_kernel_cost(self.handle, kernel, C.byref(b), C.byref(f)))
        return b.value, f.value

    def close(self):
        if self.handle:
            lib().agg_mg_hierarchy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rtree_maps(mesh, max_entries=8, n_maps=None):
    """agg_rtree_agglomerate: the nested agglomeration maps of the mesh's
    R*-tree (all node levels when n_maps is None), as int32 arrays."""
    levels = C.c_int()
    _check(lib().agg_rtree_agglomerate(mesh.handle, max_entries, 0, None, None, C.byref(levels)))
    n_maps = levels.value if n_maps is None else n_maps
    bufs = [np.full(mesh.n_elements, -1, dtype=np.int32) for _ in range(n_maps)]
    ptrs = (C.POINTER(C.c_int32) * max(n_maps, 1))(*[b.ctypes.data_as(C.POINTER(C.c_int32)) for b in bufs])
    units = (C.c_int64 * max(n_maps, 1))()
    _check(lib().agg_rtree_agglomerate(mesh.handle, max_entries, n_maps, ptrs, units, C.byref(levels)))
    sizes = [mesh.n_elements] + [units[k] for k in range(n_maps)]
    return [bufs[k][:sizes[k]].copy() for k in range(n_maps)]


def n_gates(d: dict) -> int:
    """Gating variables per DoF of the model (w holds n_gates rows of n DoFs)."""
    return 3 if int(d["model"]) == AGG_BUENO_OROVIO else 1


def ionic_params(d: dict) -> IonicParams:
    bo = BuenoOrovioParams(*[d[f] for f in BO_FIELDS]) if int(d["model"]) == AGG_BUENO_OROVIO \
        else BuenoOrovioParams()
    return IonicParams(int(d["model"]), d.get("k", 0.0), d.get("a", 0.0), d.get("eps", 0.0), d.get("gamma", 0.0),
                       d.get("mu1", 0.0), d.get("mu2", 0.0), bo)


def ionic_update(prm: dict, dt: float, u, w, stream=None):
    """agg_ionic_update; w holds n_gates(prm) gate rows of u.numel() values."""
    if w.numel() != n_gates(prm) * u.numel():
        raise ValueError("w must hold n_gates * n values")
    p = ionic_params(prm)
    _check(lib().agg_ionic_update(C.byref(p), dt, u.numel(), C.c_void_p(_dptr(u)), C.c_void_p(_dptr(w)),
                                  C.c_void_p(_stream(stream))))


class Monodomain:
    """agg_monodomain_create / agg_monodomain_step on a hierarchy."""

    def __init__(self, hier: Hierarchy, dt, ionic: dict, iapp_mask=None, iapp_value=1.0, iapp_steps=5,
                 rtol=1e-8, atol=0.0, max_it=500, flexible=False, chi_m=1.0, c_m=1.0, scheme=0):
        self._mask = iapp_mask
        o = SimOpts(dt, chi_m, c_m, ionic_params(ionic), C.c_void_p(_dptr(iapp_mask)) if iapp_mask is not None
                    else None, iapp_value, iapp_steps, PCGOpts(rtol, atol, max_it, int(flexible)), int(scheme))
        h = C.c_void_p()
        _check(lib().agg_monodomain_create(hier.handle, C.byref(o), C.byref(h)))
        self.handle = h
        self.hier = hier
        self.n_gates = n_gates(ionic)

    def step(self, u, w, n_steps=1, stream=None, iters=True):
        """Advance in place; w holds n_gates rows of u.numel() gate values."""
        if w.numel() != self.n_gates * u.numel():
            raise ValueError("w must hold n_gates * n_dofs values")
        its = (C.c_int * n_steps)() if iters else None
        _check(lib().agg_monodomain_step(self.handle, n_steps, C.c_void_p(_dptr(u)), C.c_void_p(_dptr(w)),
                                         its, C.c_void_p(_stream(stream))))
        return list(its) if iters else None

    def set_clock(self, step):
        _check(lib().agg_monodomain_set_clock(self.handle, step))

    def adjoint_step(self, u_n, w_n, u_np1, ubar, wbar, grad_logD, stream=None):
        """agg_monodomain_adjoint_step: ubar, wbar updated in place, grad_logD accumulated."""
        _check(lib().agg_monodomain_adjoint_step(self.handle, C.c_void_p(_dptr(u_n)), C.c_void_p(_dptr(w_n)),
                                                 C.c_void_p(_dptr(u_np1)), C.c_void_p(_dptr(ubar)),
                                                 C.c_void_p(_dptr(wbar)), C.c_void_p(_dptr(grad_logD)),
                                                 C.c_void_p(_stream(stream))))

    def close(self):
        if self.handle:
            lib().agg_monodomain_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
