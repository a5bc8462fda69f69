"""Pins of the oracle's reference element against closed forms."""
import math

import numpy as np
import pytest

from oracle import refelem as re


@pytest.mark.parametrize("p,interior", [
    (1, []),
    (2, [0.0]),
    (3, [-1 / math.sqrt(5), 1 / math.sqrt(5)]),
    (4, [-math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7)]),
])
def test_gll_closed_forms(p, interior):
    # GLL nodes on [-1, 1]: endpoints plus the roots of P_p' (closed forms)
    expect = 0.5 * (np.array([-1.0] + interior + [1.0]) + 1.0)
    np.testing.assert_allclose(re.gll_nodes(p), expect, atol=1e-15)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_gauss_exact_on_monomials(q):
    x, w = re.gauss_rule(q)
    for k in range(2 * q):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
    # not exact at degree 2q
    assert abs(np.sum(w * x ** (2 * q)) - 1.0 / (2 * q + 1)) > 1e-8


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_kronecker_unity_and_derivative(p):
    nodes = re.gll_nodes(p)
    val, der = re.lagrange_1d(nodes, nodes)
    np.testing.assert_allclose(val, np.eye(p + 1), atol=1e-14)
    x = np.linspace(0, 1, 17)
    val, der = re.lagrange_1d(nodes, x)
    np.testing.assert_allclose(val.sum(0), 1.0, atol=1e-13)
    np.testing.assert_allclose(der.sum(0), 0.0, atol=1e-11)
    # interpolation of x^p and its derivative is exact
    f = nodes ** p
    np.testing.assert_allclose(f @ val, x ** p, atol=1e-13)
    np.testing.assert_allclose(f @ der, p * x ** (p - 1), atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_tensor_basis_and_multilinear(dim):
    p = 2
    xi = np.random.default_rng(0).uniform(size=(7, dim))
    phi, grad = re.tensor_basis(p, dim, xi)
    np.testing.assert_allclose(phi.sum(0), 1.0, atol=1e-13)
    np.testing.assert_allclose(grad.sum(0), 0.0, atol=1e-11)
    # nodal interpolation of q(x) = x0^2 x_last + x1 reproduces q and grad q
    nodes = re.tensor_points(re.gll_nodes(p), dim)
    q = lambda y: y[:, 0] ** 2 * y[:, -1] + y[:, 1]
    np.testing.assert_allclose(q(nodes) @ phi, q(xi), atol=1e-13)
    gx = q(nodes) @ grad[:, :, 0]
    np.testing.assert_allclose(gx, 2 * xi[:, 0] * xi[:, -1], atol=1e-12)
    N, dN = re.multilinear_shape(dim, xi)
    np.testing.assert_allclose(N.sum(1), 1.0, atol=1e-15)
    corners = np.array([[(c >> k) & 1 for k in range(dim)] for c in range(2 ** dim)], float)
    np.testing.assert_allclose(N @ corners, xi, atol=1e-15)
    np.testing.assert_allclose(np.einsum("qvl,vk->qkl", dN, corners),
                               np.broadcast_to(np.eye(dim), (7, dim, dim)), atol=1e-15)
