"""Reference element of the DG space V_h^p (Section 3): tensor-product
Lagrange basis on Gauss-Lobatto (GLL) nodes of the unit interval, and the
Gauss-Legendre quadrature used for all volume and face integrals.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Pins (tests/test_oracle_refelem.py): GLL nodes against their closed forms for
p = 1..4, Gauss rule exactness on monomials, Kronecker property, partition of
unity, exact derivatives of interpolated polynomials.
"""
import itertools

import numpy as np
from numpy.polynomial import legendre as L


def gll_nodes(p: int) -> np.ndarray:
    """Gauss-Lobatto nodes of degree p on [0, 1]: the two end points and the
    p-1 roots of P_p' (derivative of the Legendre polynomial), ascending."""
    if p < 1:
        raise ValueError("p >= 1")
    coef = np.zeros(p + 1)
    coef[p] = 1.0
    interior = np.sort(np.real(L.legroots(L.legder(coef)))) if p >= 2 else np.zeros(0)
    t = np.concatenate([[-1.0], interior, [1.0]])
    return 0.5 * (t + 1.0)


def gauss_rule(q: int):
    """q-point Gauss-Legendre rule on [0, 1] (exact for degree 2q-1)."""
    t, w = L.leggauss(q)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange_1d(nodes: np.ndarray, x: np.ndarray):
    """Values and derivatives of the Lagrange polynomials through `nodes` at x.

    Returns (val, der) with shape (len(nodes), len(x)):
      l_i(x)  = prod_{m != i} (x - x_m) / (x_i - x_m)
      l_i'(x) = sum_{k != i} 1/(x_i - x_k) prod_{m != i,k} (x - x_m)/(x_i - x_m)
    """
    x = np.asarray(x, dtype=np.float64)
    n = len(nodes)
    val = np.ones((n, x.size))
    der = np.zeros((n, x.size))
    for i in range(n):
        for m in range(n):
            if m != i:
                val[i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
        for k in range(n):
            if k == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[i] - nodes[k]))
            for m in range(n):
                if m != i and m != k:
                    term *= (x - nodes[m]) / (nodes[i] - nodes[m])
            der[i] += term
    return val, der


def multi_indices(dim: int, n: int) -> np.ndarray:
    """Tensor multi-indices (i_0, ..., i_{d-1}) of the flat index
    i = i_0 + n i_1 + n^2 i_2 (x fastest), shape (n**dim, dim)."""
    out = [tuple(reversed(t)) for t in itertools.product(range(n), repeat=dim)]
    return np.array(out, dtype=np.int64)


def tensor_points(x1d: np.ndarray, dim: int) -> np.ndarray:
    """Tensor grid of 1D points, flat index x fastest, shape (n**dim, dim)."""
    idx = multi_indices(dim, len(x1d))
    return x1d[idx]


def tensor_weights(w1d: np.ndarray, dim: int) -> np.ndarray:
    idx = multi_indices(dim, len(w1d))
    return np.prod(w1d[idx], axis=1)


def tensor_basis(p: int, dim: int, xi: np.ndarray):
    """Tensor Lagrange basis of Q_p on GLL nodes at reference points xi (Q, dim).

    Returns phi (B, Q) and grad (B, Q, dim) with B = (p+1)**dim and
    phi_i(xi) = prod_k l_{i_k}(xi_k).
    """
    nodes = gll_nodes(p)
    idx = multi_indices(dim, p + 1)
    Q = xi.shape[0]
    vals, ders = [], []
    for k in range(dim):
        v, d = lagrange_1d(nodes, xi[:, k])
        vals.append(v)
        ders.append(d)
    B = idx.shape[0]
    phi = np.ones((B, Q))
    grad = np.ones((B, Q, dim))
    for k in range(dim):
        phi *= vals[k][idx[:, k]]
        for l in range(dim):
            grad[:, :, l] *= (ders[k] if k == l else vals[k])[idx[:, k]]
    return phi, grad


def multilinear_shape(dim: int, xi: np.ndarray):
    """Shape functions of the multilinear element map at xi (Q, dim).

    Corner c has reference coordinates (c>>k)&1. Returns N (Q, 2**dim) and
    dN (Q, 2**dim, dim)."""
    Q = xi.shape[0]
    V = 2 ** dim
    N = np.ones((Q, V))
    dN = np.ones((Q, V, dim))
    for c in range(V):
        for k in range(dim):
            bit = (c >> k) & 1
            f = xi[:, k] if bit else 1.0 - xi[:, k]
            df = 1.0 if bit else -1.0
            N[:, c] *= f
            for l in range(dim):
                dN[:, c, l] *= df if l == k else f
    return N, dN
