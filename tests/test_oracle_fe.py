"""Pins of the oracle's 1D bases, quadrature and Q1 map against textbook facts."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import fe


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_gauss_lobatto_nodes_are_endpoints_and_roots_of_dPk(k):
    nodes = fe.gauss_lobatto_nodes(k)
    roots = np.sort(npleg.Legendre.basis(k).deriv().roots().real)
    expect = np.concatenate([[0.0], 0.5 * (roots + 1.0), [1.0]])
    np.testing.assert_allclose(nodes, expect, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_legendre_matches_library_and_moments(n):
    x, w = fe.gauss_legendre(n)
    t, wl = npleg.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (t + 1.0), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * wl, atol=1e-15)
    for j in range(2 * n):          # exact up to degree 2n-1
        assert abs(np.sum(w * x ** j) - 1.0 / (j + 1)) < 1e-14
    assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-8


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_lagrange_cardinal_partition_of_unity_and_derivative(k):
    nodes = fe.gauss_lobatto_nodes(k)
    L, dL = fe.lagrange(nodes, nodes)
    np.testing.assert_allclose(L, np.eye(k + 1), atol=1e-14)
    x = np.linspace(-0.3, 1.3, 37)
    L, dL = fe.lagrange(nodes, x)
    np.testing.assert_allclose(L.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(dL.sum(1), 0.0, atol=1e-12)
    for j in range(k + 1):          # reproduces monomials up to degree k
        np.testing.assert_allclose(L @ nodes ** j, x ** j, atol=1e-12)
        np.testing.assert_allclose(dL @ nodes ** j, j * x ** max(j - 1, 0) * (j > 0), atol=1e-11)
    h = 1e-6
    Lp, _ = fe.lagrange(nodes, x + h)
    Lm, _ = fe.lagrange(nodes, x - h)
    np.testing.assert_allclose(dL, (Lp - Lm) / (2 * h), atol=1e-7)


@pytest.mark.parametrize("dim", [2, 3])
def test_q1_shape_partition_and_gradient(dim):
    rng = np.random.default_rng(3)
    xi = rng.random((20, dim))
    N, dN = fe.q1_shape(dim, xi)
    np.testing.assert_allclose(N.sum(1), 1.0, atol=1e-15)
    corners = np.array([[(v >> d) & 1 for d in range(dim)] for v in range(2 ** dim)], float)
    np.testing.assert_allclose(N @ corners, xi, atol=1e-15)      # F = identity on the unit cell
    np.testing.assert_allclose(np.einsum("pvb,va->pab", dN, corners),
                               np.broadcast_to(np.eye(dim), (20, dim, dim)), atol=1e-15)


@pytest.mark.parametrize("k,dim", [(1, 2), (3, 2), (2, 3), (4, 3)])
def test_tensor_basis_interpolates_tensor_polynomials(k, dim):
    rng = np.random.default_rng(1)
    pts = rng.random((30, dim))
    val, grad = fe.tensor_basis(k, dim, pts)
    nodes = fe.gauss_lobatto_nodes(k)
    npts = nodes[fe.multi_indices(k + 1, dim)]
    e = rng.integers(0, k + 1, size=dim)               # x^e0 y^e1 (z^e2) lies in Q_k
    f = lambda p: np.prod(p ** e, axis=1)
    np.testing.assert_allclose(val @ f(npts), f(pts), atol=1e-12)
    for a in range(dim):
        ea = e.copy()
        ea[a] -= 1
        g = e[a] * np.prod(pts ** np.maximum(ea, 0), axis=1) * (e[a] > 0)
        np.testing.assert_allclose(grad[:, :, a] @ f(npts), g, atol=1e-11)
