"""Agglomeration-based multigrid preconditioned CG (Sections 5 and 6).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Steps, in the paper's order:
  * Nested levels T_0 (the mesh) ... T_{L-1}; level l+1 units are
    agglomerates of level-l units given by element->agglomerate maps
    (Section 4 builds them with R-trees; here they are inputs).
  * Coarse basis: the tensor Q_p Lagrange (GLL) basis of the axis-aligned
    bounding box B_K of each agglomerate, restricted to K (Section 5.1).
  * Prolongation P_{l+1}^l: the embedding of the coarse space into the fine
    one, evaluated by nodal interpolation at the nodal points of every level-l
    unit; restriction R = P^T (Section 5.1, Section 6 "natural embedding").
  * Inherited (Galerkin) coarse operators A_{l+1} = P^T A_l P
    (Eq. inherited_matrices, Algorithm 3).
  * Smoother: Chebyshev-accelerated (block-)Jacobi of degree 3, bounds from a
    Lanczos estimate (Section 6, first paragraph).
  * One V-cycle per PCG iteration; coarsest level solved directly
    (dense Cholesky); PCG on A0 warm-started from the previous time step
    (Section 6, first paragraph; Section 3.1).

Readings (the paper does not fix these):
  * Nodal interpolation at the fine element's mapped GLL nodes defines P on
    level 0; on levels >= 1 the spaces are exactly nested.
  * Smoother blocks: the b x b diagonal blocks of A_l (block Jacobi);
    block_jacobi=False gives the paper's point Jacobi.
  * Chebyshev: one degree-3 application before and one after the coarse
    correction (3 residual evaluations each). Bounds: lambda_hat = largest
    Ritz value of D^{-1} A_l after 12 Lanczos steps (D-inner product, start
    vector v_i = sin(i+1)), lambda_max = 1.2 lambda_hat,
    lambda_min = lambda_max / 20.
  * PCG stops when ||r_k||_2 <= rtol ||r_0||_2 (relative form of the
    paper's eight-orders-of-magnitude reduction); the iteration count is the
    number of products A0 p.

Pins (tests/test_oracle_multigrid.py): P reproduces Q_p (Cartesian) and P_p
(jittered) polynomials, P 1 = 1, R = P^T; A_{l+1} symmetric, SPD for c > 0,
A_{l+1} 1 = 0 for c = 0; D^{-1} D = I; Chebyshev error propagator equal to
the scaled Chebyshev polynomial T_3 from an eigen-decomposition; Lanczos
estimate equal to the exact generalized eigenvalue when steps >= n; V-cycle
symmetric and positive; one level -> B = A^{-1} and PCG in one iteration;
PCG against a dense direct solve.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import direct_coarse
from . import refelem as re
from .sipg import nodal_points


# ---------------------------------------------------------------- levels
def level1_boxes(vertices, elements, amap):
    """Bounding box of every level-1 agglomerate: min/max over the vertices of
    its fine elements. Returns lo, hi (N_1, d)."""
    X = vertices[elements]                       # (E, V, d)
    emin = X.min(axis=1)
    emax = X.max(axis=1)
    n1 = int(amap.max()) + 1
    lo = np.full((n1, vertices.shape[1]), np.inf)
    hi = np.full((n1, vertices.shape[1]), -np.inf)
    np.minimum.at(lo, amap, emin)
    np.maximum.at(hi, amap, emax)
    return lo, hi


def coarser_boxes(lo, hi, amap):
    """Boxes of level-(l+1) agglomerates from the boxes of their children."""
    n = int(amap.max()) + 1
    clo = np.full((n, lo.shape[1]), np.inf)
    chi = np.full((n, lo.shape[1]), -np.inf)
    np.minimum.at(clo, amap, lo)
    np.maximum.at(chi, amap, hi)
    return clo, chi


def box_nodal_points(lo, hi, p):
    """GLL nodes of Q_p(B_K) mapped affinely onto each box, (N, B, d)."""
    dim = lo.shape[1]
    xi = re.tensor_points(re.gll_nodes(p), dim)
    return lo[:, None, :] + xi[None, :, :] * (hi - lo)[:, None, :]


def box_basis(lo, hi, p, y):
    """Values of the Q_p(B_K) Lagrange basis of box (lo, hi) at points y.

    lo, hi (n, d); y (n, m, d) -> (n, m, B):
      phi_j^K(y) = prod_k l_{j_k}((y_k - lo_k) / (hi_k - lo_k))."""
    n, m, dim = y.shape
    nodes = re.gll_nodes(p)
    idx = re.multi_indices(dim, p + 1)
    eta = (y - lo[:, None, :]) / (hi - lo)[:, None, :]
    out = np.ones((n, m, idx.shape[0]))
    for k in range(dim):
        v, _ = re.lagrange_1d(nodes, eta[:, :, k].ravel())      # (p+1, n*m)
        v = v.reshape(p + 1, n, m).transpose(1, 2, 0)            # (n, m, p+1)
        out *= v[:, :, idx[:, k]]
    return out


def prolongation(y_fine, amap, lo_c, hi_c, p):
    """P_{l+1}^l as a sparse (N_l B) x (N_{l+1} B) matrix:
    P[(e, i), (K, j)] = phi_j^K(y_{e,i}) for K = amap[e], zero otherwise."""
    n_f, B, _ = y_fine.shape
    blocks = box_basis(lo_c[amap], hi_c[amap], p, y_fine)       # (n_f, B, B)
    ii, jj = np.meshgrid(np.arange(B), np.arange(B), indexing="ij")
    rows = (np.arange(n_f)[:, None, None] * B + ii).ravel()
    cols = (amap.astype(np.int64)[:, None, None] * B + jj).ravel()
    n_c = int(amap.max()) + 1
    return sp.csr_matrix((blocks.ravel(), (rows, cols)), shape=(n_f * B, n_c * B))


def galerkin(A, P):
    """Inherited coarse operator A_{l+1} = P^T A_l P (Eq. inherited_matrices)."""
    return (P.T @ (A @ P)).tocsr()


def diagonal_blocks(A, B):
    """The b x b diagonal blocks of A, (N, B, B)."""
    n = A.shape[0] // B
    Ab = sp.bsr_matrix(A, blocksize=(B, B))
    rows = np.repeat(np.arange(n), np.diff(Ab.indptr))
    sel = Ab.indices == rows
    out = np.zeros((n, B, B))
    out[rows[sel]] = Ab.data[sel]
    return out


def block_apply(blocks, x):
    """y_e = blocks_e x_e for a block-diagonal matrix."""
    n, B, _ = blocks.shape
    return np.einsum("eij,ej->ei", blocks, x.reshape(n, B)).ravel()


def lanczos_max_eig(A, Dblocks, steps=12):
    """Largest Ritz value of D^{-1} A after `steps` Lanczos steps in the
    D-inner product <x, y>_D = x^T D y, started from v_i = sin(i+1)."""
    n = A.shape[0]
    m = min(steps, n)
    Dinv = np.linalg.inv(Dblocks)
    v = np.sin(np.arange(1, n + 1, dtype=np.float64))
    v /= np.sqrt(v @ block_apply(Dblocks, v))
    v_prev = np.zeros(n)
    beta = 0.0
    alphas, betas = [], []
    for j in range(m):
        Av = A @ v
        alpha = Av @ v
        w = block_apply(Dinv, Av) - alpha * v - beta * v_prev
        alphas.append(alpha)
        if j == m - 1:
            break
        beta = np.sqrt(max(w @ block_apply(Dblocks, w), 0.0))
        if beta == 0.0:
            break
        betas.append(beta)
        v_prev, v = v, w / beta
    k = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    return float(np.linalg.eigvalsh(T).max())


@dataclass
class Level:
    A: sp.csr_matrix
    n_units: int
    B: int
    Dblocks: Optional[np.ndarray] = None
    Dinv: Optional[np.ndarray] = None
    lam_max: float = 0.0
    lam_min: float = 0.0
    P: Optional[sp.csr_matrix] = None        # prolongation from level l+1 to l
    lo: Optional[np.ndarray] = None
    hi: Optional[np.ndarray] = None


@dataclass
class Hierarchy:
    levels: List[Level]
    chol: Optional[tuple] = None             # scipy cho_factor of the coarsest A
    degree: int = 3
    info: dict = field(default_factory=dict)

    @property
    def n_levels(self):
        return len(self.levels)


def point_jacobi_blocks(A, B):
    """Diagonal of A as 1 x 1 blocks inside B x B block storage."""
    d = A.diagonal()
    n = A.shape[0] // B
    out = np.zeros((n, B, B))
    out[:, np.arange(B), np.arange(B)] = d.reshape(n, B)
    return out


def build_hierarchy(disc, mass_coeff, maps, block_jacobi=True, lanczos_steps=12,
                    safety=1.2, cheb_range=20.0, degree=3, direct=None):
    """Algorithm 3 (GenerateCoarserOperators) plus the smoother set-up.
    direct = dict(D=conductivity (E, d, d), c_pen=C_pen[, quad_extra=1])
    assembles the coarse operators on the agglomerates instead of the
    Galerkin products (the non-inherited operators of Section 5.1,
    oracle.direct_coarse); None keeps the inherited ones."""
    A0 = disc.A0(mass_coeff)
    p, B = disc.p, disc.B
    levels = [Level(A=A0, n_units=disc.n_elements, B=B)]
    y = nodal_points(disc.vertices, disc.elements, p)
    lo = hi = None
    unit = np.arange(disc.n_elements, dtype=np.int64)      # fine element -> unit of the current level
    for l, amap in enumerate(maps):
        amap = np.asarray(amap, dtype=np.int64)
        if l == 0:
            lo, hi = level1_boxes(disc.vertices, disc.elements, amap)
        else:
            lo, hi = coarser_boxes(lo, hi, amap)
        P = prolongation(y, amap, lo, hi, p)
        levels[l].P = P
        unit = amap[unit]
        if direct is None:
            Ac = galerkin(levels[l].A, P)
        else:
            Ac = direct_coarse.level_operator(disc.vertices, disc.elements, direct["D"], p, mass_coeff,
                                              direct["c_pen"], unit, lo, hi, direct.get("quad_extra", 1))
        levels.append(Level(A=Ac, n_units=int(amap.max()) + 1, B=B, lo=lo, hi=hi))
        y = box_nodal_points(lo, hi, p)
    for lev in levels[:-1]:
        Db = diagonal_blocks(lev.A, B) if block_jacobi else point_jacobi_blocks(lev.A, B)
        if not block_jacobi:
            Dinv = np.zeros_like(Db)
            dd = np.einsum("eii->ei", Db)
            Dinv[:, np.arange(B), np.arange(B)] = 1.0 / dd
        else:
            Dinv = np.linalg.inv(Db)
        lev.Dblocks, lev.Dinv = Db, Dinv
        lam = lanczos_max_eig(lev.A, Db, lanczos_steps)
        lev.lam_max = safety * lam
        lev.lam_min = lev.lam_max / cheb_range
    Ac = levels[-1].A.toarray()
    chol = sla.cho_factor(Ac, lower=True)
    return Hierarchy(levels, chol, degree)


# ---------------------------------------------------------------- smoother / cycle
def chebyshev(A, Dinv, b, x, lam_min, lam_max, degree=3, x_is_zero=False):
    """Chebyshev-accelerated Jacobi iteration of the given degree on A x = b
    (the three-term recurrence of Saad, Iterative Methods, Alg. 12.1, applied
    to D^{-1} A on [lam_min, lam_max])."""
    theta = 0.5 * (lam_max + lam_min)
    delta = 0.5 * (lam_max - lam_min)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b.copy() if x_is_zero else b - A @ x
    d = block_apply(Dinv, r) / theta
    x = d.copy() if x_is_zero else x + d
    for _ in range(1, degree):
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * block_apply(Dinv, b - A @ x)
        x = x + d
        rho = rho_new
    return x


def vcycle(h: Hierarchy, r, l=0):
    """One V-cycle on level l applied to residual r (returns the correction)."""
    if l == h.n_levels - 1:
        return sla.cho_solve(h.chol, r)
    lev = h.levels[l]
    e = chebyshev(lev.A, lev.Dinv, r, None, lev.lam_min, lev.lam_max, h.degree, x_is_zero=True)
    rc = lev.P.T @ (r - lev.A @ e)
    e = e + lev.P @ vcycle(h, rc, l + 1)
    e = chebyshev(lev.A, lev.Dinv, r, e, lev.lam_min, lev.lam_max, h.degree)
    return e


@dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    r0_norm: float
    r_norm: float
    converged: bool
    history: list


def pcg(A, b, x0, precond, rtol=1e-8, max_it=500):
    """Preconditioned conjugate gradients; stops when ||r|| <= rtol ||r0||."""
    x = x0.copy()
    r = b - A @ x
    r0 = float(np.linalg.norm(r))
    hist = [r0]
    if r0 == 0.0:
        return PCGResult(x, 0, 0.0, 0.0, True, hist)
    z = precond(r)
    p = z.copy()
    rho = float(r @ z)
    it = 0
    rn = r0
    while it < max_it:
        q = A @ p
        alpha = rho / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rn = float(np.linalg.norm(r))
        hist.append(rn)
        if rn <= rtol * r0:
            return PCGResult(x, it, r0, rn, True, hist)
        z = precond(r)
        rho_new = float(r @ z)
        p = z + (rho_new / rho) * p
        rho = rho_new
    return PCGResult(x, it, r0, rn, False, hist)
