"""Seeded synthetic inputs for the SIPG-DG monodomain solver.

This module is shared by the CUDA path, the oracle, the tests and the
benchmark. It holds no arithmetic of the method itself: it only builds the
inputs the method consumes (mesh vertices and connectivity, per-element
conductivity tensors, element->agglomerate maps, stimulus masks, conductivity
scales and sensor points), from numpy's PCG64 generator with fixed seeds.

Conventions (shared by every consumer):
  * Elements are quadrilaterals (d=2) or hexahedra (d=3) with a multilinear
    map. Corner c of an element has reference coordinates (c & 1, c >> 1 & 1,
    c >> 2 & 1): lexicographic, x fastest.
  * Meshes are conforming: neighbouring elements share vertex ids.
  * Conductivity is one symmetric d x d tensor per element,
    D = sigma_t I + (sigma_l - sigma_t) f f^T, i.e. the fibre/sheet/normal
    decomposition of the monodomain model (Section 2.2) with sigma_n = sigma_t.
  * An agglomeration map of level l sends each level-l unit to a level-(l+1)
    agglomerate id in [0, N_{l+1}).

Workload shapes follow the paper's experiments: the 2D unit-square runs
(Section 6.1), hexahedral 3D runs (Sections 6.2-6.3) and a ventricle-like
shell. The paper's own meshes (idealised and CAD left ventricles) are not
available; the generators below are synthetic stand-ins of the same kind.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Mesh:
    dim: int
    vertices: np.ndarray            # (n_vertices, dim) float64
    elements: np.ndarray            # (n_elements, 2**dim) int64, lexicographic corners
    grid_shape: tuple               # logical element grid (n_x, n_y[, n_z])
    kind: str = "box"               # "box" or "shell"

    @property
    def n_elements(self) -> int:
        return int(self.elements.shape[0])

    def centroids(self) -> np.ndarray:
        return self.vertices[self.elements].mean(axis=1)


def box_mesh(dim: int, n: int, jitter: float = 0.0, seed: Optional[int] = None) -> Mesh:
    """Uniform n^dim grid on the unit square/cube, element index x fastest.

    Interior vertices are moved by independent U(-jitter*h, jitter*h) offsets in
    every coordinate (numpy PCG64, `seed`); boundary vertices stay fixed so the
    domain is exactly [0,1]^dim.
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    h = 1.0 / n
    m = n + 1
    idx = np.indices((m,) * dim).reshape(dim, -1)[::-1]   # idx[0] = x index (fastest)
    verts = (idx.T.astype(np.float64)) * h
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        off = rng.uniform(-jitter * h, jitter * h, size=verts.shape)
        interior = np.all((idx > 0) & (idx < n), axis=0)
        verts = verts + off * interior[:, None]
    # elements
    eidx = np.indices((n,) * dim).reshape(dim, -1)[::-1]   # eidx[0] = x index
    corners = []
    for c in range(2 ** dim):
        off = [(c >> k) & 1 for k in range(dim)]
        vid = np.zeros(eidx.shape[1], dtype=np.int64)
        stride = 1
        for k in range(dim):
            vid += (eidx[k] + off[k]) * stride
            stride *= m
        corners.append(vid)
    elems = np.stack(corners, axis=1)
    return Mesh(dim, verts, elems, (n,) * dim, "box")


def shell_mesh(n_circ: int = 128, n_long: int = 96, n_trans: int = 16,
               inner=(2.5, 2.5, 4.5), thickness: float = 1.0,
               v_range=(0.5 * math.pi, 0.97 * math.pi)) -> Mesh:
    """Truncated prolate-ellipsoidal shell, hex-mapped, periodic in the
    circumferential direction (shared vertex ids at the seam).

    Parameters s (transmural, 0 = endocardium), u (circumferential) and v
    (longitudinal, v = pi/2 is the base plane z = 0, larger v towards the apex):
      x = a(s) sin v cos u,  y = a(s) sin v sin u,  z = c(s) cos v,
      a(s) = inner[0] + s*thickness, c(s) = inner[2] + s*thickness.
    Logical element grid (n_circ, n_long, n_trans) with the circumferential
    index fastest.
    """
    nu, nv, ns = n_circ, n_long, n_trans
    us = np.arange(nu) * (2 * math.pi / nu)
    vs = np.linspace(v_range[0], v_range[1], nv + 1)
    ss = np.linspace(0.0, 1.0, ns + 1)
    S, V, U = np.meshgrid(ss, vs, us, indexing="ij")     # (ns+1, nv+1, nu), u fastest
    a = inner[0] + S * thickness
    b = inner[1] + S * thickness
    c = inner[2] + S * thickness
    X = a * np.sin(V) * np.cos(U)
    Y = b * np.sin(V) * np.sin(U)
    Z = c * np.cos(V)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(iu, iv, is_):
        return (is_ * (nv + 1) + iv) * nu + (iu % nu)

    ie = np.indices((ns, nv, nu)).reshape(3, -1)          # [s, v, u], u fastest
    is_, iv, iu = ie[0], ie[1], ie[2]
    # reference axes: xi_0 <-> u, xi_1 <-> v, xi_2 <-> s; orientation fixed below
    corners = []
    for cidx in range(8):
        du, dv, ds = cidx & 1, (cidx >> 1) & 1, (cidx >> 2) & 1
        corners.append(vid(iu + du, iv + dv, is_ + ds))
    elems = np.stack(corners, axis=1).astype(np.int64)
    # right-handed reference frame: swap xi_0/xi_1 if the signed volume is negative
    e0 = verts[elems[0]]
    j = np.stack([e0[1] - e0[0], e0[2] - e0[0], e0[4] - e0[0]], axis=1)
    if np.linalg.det(j) < 0:
        perm = [0, 2, 1, 3, 4, 6, 5, 7]
        elems = elems[:, perm]
    return Mesh(3, verts, elems, (nu, nv, ns), "shell")


# --------------------------------------------------------------------------
# conductivity
# --------------------------------------------------------------------------
def conductivity_from_fibres(fibres: np.ndarray, sigma_l: float, sigma_t: float) -> np.ndarray:
    """D = sigma_t I + (sigma_l - sigma_t) f f^T per element (unit fibres f)."""
    f = fibres / np.linalg.norm(fibres, axis=1, keepdims=True)
    d = f.shape[1]
    return sigma_t * np.eye(d)[None] + (sigma_l - sigma_t) * f[:, :, None] * f[:, None, :]


def isotropic_conductivity(n_elements: int, dim: int, sigma: float) -> np.ndarray:
    return np.broadcast_to(sigma * np.eye(dim), (n_elements, dim, dim)).copy()


def planar_fibres(n_elements: int, angle_deg) -> np.ndarray:
    """Fibres in the x-y plane at the given angle(s) from the x axis (2D)."""
    a = np.deg2rad(np.broadcast_to(np.asarray(angle_deg, dtype=np.float64), (n_elements,)))
    return np.stack([np.cos(a), np.sin(a)], axis=1)


def rotating_fibres_z(centroids: np.ndarray, top_deg=60.0, bottom_deg=-60.0) -> np.ndarray:
    """3D fibres in planes z = const, angle linear in z from +60 (z=0) to -60 (z=1)."""
    z = centroids[:, 2]
    a = np.deg2rad(top_deg + (bottom_deg - top_deg) * z)
    return np.stack([np.cos(a), np.sin(a), np.zeros_like(a)], axis=1)


def shell_helix_fibres(mesh: Mesh, endo_deg=60.0, epi_deg=-60.0,
                       inner=(2.5, 2.5, 4.5), thickness: float = 1.0,
                       v_range=(0.5 * math.pi, 0.97 * math.pi)) -> np.ndarray:
    """Helical fibres on the shell of `shell_mesh`: f = cos(a) e_circ + sin(a) e_long
    at the element's parametric centre, with the helix angle a linear in the
    transmural coordinate from endo_deg (endocardium) to epi_deg (epicardium)."""
    nu, nv, ns = mesh.grid_shape
    ie = np.indices((ns, nv, nu)).reshape(3, -1)           # [s, v, u], u fastest
    s = (ie[0] + 0.5) / ns
    v = v_range[0] + (ie[1] + 0.5) * (v_range[1] - v_range[0]) / nv
    u = (ie[2] + 0.5) * (2 * math.pi / nu)
    a = inner[0] + s * thickness
    b = inner[1] + s * thickness
    c = inner[2] + s * thickness
    ec = np.stack([-a * np.sin(v) * np.sin(u), b * np.sin(v) * np.cos(u), np.zeros_like(u)], 1)
    el = np.stack([a * np.cos(v) * np.cos(u), b * np.cos(v) * np.sin(u), -c * np.sin(v)], 1)
    ec /= np.linalg.norm(ec, axis=1, keepdims=True)
    el = el - (el * ec).sum(1, keepdims=True) * ec
    el /= np.linalg.norm(el, axis=1, keepdims=True)
    ang = np.deg2rad(endo_deg + (epi_deg - endo_deg) * s)
    return np.cos(ang)[:, None] * ec + np.sin(ang)[:, None] * el


# --------------------------------------------------------------------------
# agglomeration maps
# --------------------------------------------------------------------------
def rcb_map(points: np.ndarray, max_group: int) -> np.ndarray:
    """Recursive coordinate bisection: split each index set at the median of the
    longest axis of its points' bounding box (ties in the coordinate broken by
    index) until every set has at most `max_group` members. Groups are numbered
    depth-first, lower half first. Returns the group id of every point.
    """
    n = len(points)
    out = np.empty(n, dtype=np.int32)
    stack = [np.arange(n)]
    leaves: List[np.ndarray] = []
    while stack:
        ids = stack.pop()
        if len(ids) <= max_group:
            leaves.append(ids)
            continue
        p = points[ids]
        ext = p.max(axis=0) - p.min(axis=0)
        ax = int(np.argmax(ext))
        order = np.lexsort((ids, p[:, ax]))
        half = len(ids) // 2
        # push upper half first so the lower half is numbered first
        stack.append(ids[order[half:]])
        stack.append(ids[order[:half]])
    for g, ids in enumerate(leaves):
        out[ids] = g
    return out


def block_map(grid_shape, factors) -> tuple:
    """Structured blocking of a logical grid (x fastest): units (i, j[, k]) go to
    agglomerate (i // f0, j // f1[, k // f2]). Returns (map, coarse grid shape)."""
    dim = len(grid_shape)
    idx = np.indices(grid_shape[::-1]).reshape(dim, -1)[::-1]
    cshape = tuple((grid_shape[k] + factors[k] - 1) // factors[k] for k in range(dim))
    g = np.zeros(idx.shape[1], dtype=np.int64)
    stride = 1
    for k in range(dim):
        g += (idx[k] // factors[k]) * stride
        stride *= cshape[k]
    return g.astype(np.int32), cshape


def rcb_hierarchy(mesh: Mesh, max_group: int, n_levels: int) -> List[np.ndarray]:
    """n_levels-1 nested maps by recursive coordinate bisection, applied level by
    level to the previous level's unit centroids (mean of element centroids)."""
    maps = []
    cen = mesh.centroids()
    weights = np.ones(len(cen))
    for _ in range(n_levels - 1):
        m = rcb_map(cen, max_group)
        maps.append(m)
        nc = int(m.max()) + 1
        s = np.zeros((nc, cen.shape[1]))
        np.add.at(s, m, cen * weights[:, None])
        w = np.zeros(nc)
        np.add.at(w, m, weights)
        cen = s / w[:, None]
        weights = w
    return maps


def block_hierarchy(grid_shape, factors, n_levels: int) -> List[np.ndarray]:
    maps = []
    shape = tuple(grid_shape)
    for _ in range(n_levels - 1):
        f = tuple(min(factors[k], shape[k]) for k in range(len(shape)))
        m, shape = block_map(shape, f)
        maps.append(m)
    return maps


# --------------------------------------------------------------------------
# configurations (synthetic stand-ins for the paper's runs)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    degree: int
    conductivity: np.ndarray        # (E, d, d)
    maps: List[np.ndarray]          # n_levels-1 agglomeration maps
    penalty_mode: int               # 0: p(p+1) (paper); 1: penalty_coeff * p^2
    # The 16x16 square states 10 p^2. The other workloads leave the constant
    # open and use 4 p^2: with the paper's p(p+1) (1.5 p^2 at p = 2) the SIPG
    # stiffness is indefinite on the jittered anisotropic meshes, and on the
    # 512^2 square so is 2.5 p^2; 4 p^2 keeps it positive semidefinite there
    # (element patches of the oracle's assembly) with less stiffening of the
    # inherited coarse operators than 10 p^2.
    penalty_coeff: float
    dt: float
    n_steps: int
    ionic: Dict[str, float]
    stim_elements: np.ndarray       # bool (E,)
    iapp_value: float
    iapp_steps: int
    rtol: float
    description: str = ""
    theta: Optional[np.ndarray] = None       # per-theta-block conductivity scale
    theta_map: Optional[np.ndarray] = None   # element -> theta block
    sensors: Optional[np.ndarray] = None
    # Chebyshev smoother interval [lambda_max / cheb_range, lambda_max] (the
    # paper does not give it): 20 by default; the jittered square, whose 4x4
    # agglomerates coarsen 16:1 per level, uses 40 (measured on its 512^2
    # benchmark: 25.3 -> 23.5 PCG iterations per step; the 2x2x2-agglomerate
    # shell gets worse with a wider interval, 8 -> 10 at 40)
    cheb_range: float = 20.0

    @property
    def n_dofs(self) -> int:
        return self.mesh.n_elements * (self.degree + 1) ** self.mesh.dim

    @property
    def n_levels(self) -> int:
        return len(self.maps) + 1

    def stim_mask_nodal(self) -> np.ndarray:
        """Per-DoF 0/1 mask of the stimulated elements, element-major layout."""
        b = (self.degree + 1) ** self.mesh.dim
        return np.repeat(self.stim_elements.astype(np.float64), b)


FHN = dict(model=0, k=1.0, a=0.13, eps=0.01, gamma=0.5, mu1=0.0, mu2=0.0)
ALIEV_PANFILOV = dict(model=1, k=8.0, a=0.15, eps=0.002, gamma=0.0, mu1=0.2, mu2=0.3)
# Bueno-Orovio (Section 2.3.2, Eq. BuenoOrovio) with the values of the paper's
# appendix table (times in s, u dimensionless), its repeated rows taken once;
# uo = 0 is the reference potential of the I_so drift term (reading: see
# oracle/monodomain.py). 3 gating variables.
BUENO_OROVIO = dict(
    model=2, k=0.0, a=0.0, eps=0.0, gamma=0.0, mu1=0.0, mu2=0.0,
    tau1p=6e-2, tau1pp=1.15, tau1plus=1.4506e-3,
    tau2p=7e-2, tau2pp=2e-2, tau2plus=2.8e-1, tau2inf=7e-2,
    tau3p=2.7342e-3, tau3pp=3e-3,
    taufi=1.1e-4, tauo_p=6e-3, tauo_pp=6e-3, tauso_p=4.3e-2, tauso_pp=2e-4, tausi=2.8723e-3,
    k2=65.0, k3=2.0994, kso=2.0, winf_star=0.94,
    V1=0.3, V1m=1.5e-2, V2=1.5e-2, V2m=3e-2, V3=0.9087, Vhat=1.58, Vo=6e-3, Vso=0.65, uo=0.0)

def n_gates(ionic: dict) -> int:
    """Gating variables per DoF of an ionic model: 3 for Bueno-Orovio, else 1."""
    return 3 if ionic["model"] == 2 else 1


def resting_gates(ionic: dict) -> np.ndarray:
    """Gate values of the resting state u = 0 (one row per gate)."""
    if ionic["model"] != 2:
        return np.zeros(1)
    s_inf = 0.5 * (1.0 + np.tanh(ionic["k3"] * (0.0 - ionic["V3"])))
    return np.array([1.0, 1.0, s_inf])


def square_2d_fhn(n: int = 16, degree: int = 1) -> Workload:
    """Plain FP64 2D unit square: n x n uniform quads, DG Q_p, isotropic
    sigma = 1e-3, penalty 10 p^2/h, dt = 0.05, FitzHugh-Nagumo, stimulus 1 on
    the corner quarter for 5 steps, 2 levels of 4x4 agglomerates, rtol 1e-10,
    50 steps."""
    mesh = box_mesh(2, n)
    cen = mesh.centroids()
    maps = block_hierarchy(mesh.grid_shape, (4, 4), 2)
    return Workload(
        name=f"square2d_q{degree}_{n}x{n}", mesh=mesh, degree=degree,
        conductivity=isotropic_conductivity(mesh.n_elements, 2, 1e-3),
        maps=maps, penalty_mode=1, penalty_coeff=10.0, dt=0.05, n_steps=50,
        ionic=dict(FHN), stim_elements=np.all(cen <= 0.5, axis=1),
        iapp_value=1.0, iapp_steps=5, rtol=1e-10,
        description="2D square, FHN, Q1, 2 levels")


def jittered_square_2d(n: int = 512, degree: int = 2, n_levels: int = 4, seed: int = 1,
                       n_steps: int = 200) -> Workload:
    """2D jittered square: n x n quads, interior vertex jitter U(+-0.2h) (seed 1),
    DG Q2, fibres at 30 degrees (sigma_l = 1.2e-3, sigma_t = 2.5e-4), agglomerates
    of <= 16 units by recursive coordinate bisection per level, FHN, dt 0.05,
    rtol 1e-8."""
    mesh = box_mesh(2, n, jitter=0.2, seed=seed)
    cen = mesh.centroids()
    D = conductivity_from_fibres(planar_fibres(mesh.n_elements, 30.0), 1.2e-3, 2.5e-4)
    maps = rcb_hierarchy(mesh, 16, n_levels)
    return Workload(
        name=f"jsquare2d_q{degree}_{n}x{n}", mesh=mesh, degree=degree, conductivity=D,
        maps=maps, penalty_mode=1, penalty_coeff=4.0, dt=0.05, n_steps=n_steps,
        ionic=dict(FHN), stim_elements=np.all(cen <= 0.5, axis=1),
        iapp_value=1.0, iapp_steps=5, rtol=1e-8,
        description="2D jittered square, anisotropic 30deg fibres, FHN", cheb_range=40.0)


def jittered_cube_3d(n: int = 64, degree: int = 2, n_levels: int = 4, seed: int = 2,
                     group: int = 4, n_steps: int = 100) -> Workload:
    """3D jittered cube: n^3 hexes, jitter U(+-0.15h) (seed 2), DG Q2, fibres in
    z-planes rotating from +60 to -60 degrees, sigma_l = 1.2e-3,
    sigma_t = sigma_n = 2.5e-4, group^3 blocks per level, Aliev-Panfilov."""
    mesh = box_mesh(3, n, jitter=0.15, seed=seed)
    cen = mesh.centroids()
    D = conductivity_from_fibres(rotating_fibres_z(cen), 1.2e-3, 2.5e-4)
    maps = block_hierarchy(mesh.grid_shape, (group,) * 3, n_levels)
    return Workload(
        name=f"jcube3d_q{degree}_{n}^3", mesh=mesh, degree=degree, conductivity=D,
        maps=maps, penalty_mode=1, penalty_coeff=4.0, dt=0.05, n_steps=n_steps,
        ionic=dict(ALIEV_PANFILOV), stim_elements=np.all(cen <= 0.25, axis=1),
        iapp_value=1.0, iapp_steps=5, rtol=1e-8,
        description="3D jittered cube, rotating fibres, Aliev-Panfilov")


def cube_3d_adjoint(n: int = 48, degree: int = 3, n_levels: int = 5, seed: int = 3,
                    theta_block: int = 6, n_sensors: int = 4096, n_steps: int = 200) -> Workload:
    """3D axis-aligned cube for the adjoint: n^3 hexes, DG Q3, 2x2x2 agglomerates
    per level, per-block conductivity scales theta = exp(0.2 z), z ~ N(0,1) on
    theta_block^3 element blocks (seed 3), sensors uniform in the cube drawn
    after theta from the same generator."""
    mesh = box_mesh(3, n)
    cen = mesh.centroids()
    D = conductivity_from_fibres(rotating_fibres_z(cen), 1.2e-3, 2.5e-4)
    maps = block_hierarchy(mesh.grid_shape, (2, 2, 2), n_levels)
    tmap, tshape = block_map(mesh.grid_shape, (theta_block,) * 3)
    rng = np.random.default_rng(seed)
    theta = np.exp(0.2 * rng.standard_normal(int(np.prod(tshape))))
    sensors = rng.uniform(0.0, 1.0, size=(n_sensors, 3))
    return Workload(
        name=f"cube3d_adj_q{degree}_{n}^3", mesh=mesh, degree=degree, conductivity=D,
        maps=maps, penalty_mode=1, penalty_coeff=4.0, dt=0.05, n_steps=n_steps,
        ionic=dict(ALIEV_PANFILOV), stim_elements=np.all(cen <= 0.25, axis=1),
        iapp_value=1.0, iapp_steps=5, rtol=1e-8, theta=theta, theta_map=tmap,
        sensors=sensors, description="3D cube adjoint, theta on 6^3 blocks")


def ventricle_shell(n_circ=128, n_long=96, n_trans=16, degree: int = 2, n_levels: int = 5,
                    n_steps: int = 1000) -> Workload:
    """Truncated prolate shell (inner semi-axes 2.5/2.5/4.5, wall 1), Q2,
    transmural helix +60 -> -60 degrees, 2x2x2 agglomerates per level,
    Aliev-Panfilov, stimulus on the 4 most apical element rows."""
    mesh = shell_mesh(n_circ, n_long, n_trans)
    D = conductivity_from_fibres(shell_helix_fibres(mesh), 1.2e-3, 2.5e-4)
    maps = block_hierarchy(mesh.grid_shape, (2, 2, 2), n_levels)
    ie = np.indices((n_trans, n_long, n_circ)).reshape(3, -1)
    stim = ie[1] >= n_long - 4
    return Workload(
        name=f"shell_q{degree}_{n_circ}x{n_long}x{n_trans}", mesh=mesh, degree=degree,
        conductivity=D, maps=maps, penalty_mode=1, penalty_coeff=4.0, dt=0.05,
        n_steps=n_steps, ionic=dict(ALIEV_PANFILOV), stim_elements=stim,
        iapp_value=1.0, iapp_steps=5, rtol=1e-8,
        description="ventricle-like shell, helix fibres, Aliev-Panfilov")


def ventricle_shell_bo(n_circ=128, n_long=96, n_trans=16, degree: int = 2, n_levels: int = 5,
                       n_steps: int = 1000) -> Workload:
    """The shell of ventricle_shell in metres (inner semi-axes 2.5/2.5/4.5 cm,
    wall 1 cm) with the Bueno-Orovio model and the conductivities of the
    paper's Bueno-Orovio table (sigma_l = 1e-4, sigma_t = sigma_n = 0.5e-4
    m^2/s; sigma_n read as sigma_t), chi_m = C_m = 1, dt = 1e-4 s, stimulus
    500 /s on the 4 most apical element rows for the first 1 ms (10 steps)."""
    mesh = shell_mesh(n_circ, n_long, n_trans)
    mesh = dataclasses.replace(mesh, vertices=mesh.vertices * 0.01)
    D = conductivity_from_fibres(shell_helix_fibres(mesh), 1.0e-4, 0.5e-4)
    maps = block_hierarchy(mesh.grid_shape, (2, 2, 2), n_levels)
    ie = np.indices((n_trans, n_long, n_circ)).reshape(3, -1)
    stim = ie[1] >= n_long - 4
    return Workload(
        name=f"shell_bo_q{degree}_{n_circ}x{n_long}x{n_trans}", mesh=mesh, degree=degree,
        conductivity=D, maps=maps, penalty_mode=1, penalty_coeff=4.0, dt=1e-4,
        n_steps=n_steps, ionic=dict(BUENO_OROVIO), stim_elements=stim,
        iapp_value=500.0, iapp_steps=10, rtol=1e-8,
        description="ventricle-like shell in metres, helix fibres, Bueno-Orovio")


def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) test vector."""
    return np.random.default_rng(seed).standard_normal(n)
