"""Pins of the oracle's assembled operators and load vectors.

What the mathematics fixes, independently of how the oracle computes it:
symmetry, constants in the kernel of the Neumann Laplacian, the patch test,
the exact energy of linear fields, rigid-body modes in the kernel of the
elasticity operator (Sec. 4.4, Eq. rbm), invariance under renumbering and
re-orientation of the mesh, and O(h^(k+1)) L2 convergence on a manufactured
solution.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assembly, dofs, fe
from tests.oracle_meshes import box_level, scramble


def _assemble(lv, k, ncomp=1, lame=(1.0, 1.0)):
    node_of, nn, oc, ol = dofs.number_dofs(lv.cells, k, lv.dim)
    elem = assembly.element_matrices(lv.vertices, lv.cells, k, lv.dim, ncomp, lame)
    A = assembly.assemble(elem, node_of, nn, ncomp)
    pts = dofs.support_points(lv.vertices, lv.cells, oc, ol, k, lv.dim)
    return A, pts, node_of, nn


CASES = [((4, 3), 1), ((3, 3), 2), ((3, 2), 3), ((2, 2), 4), ((3, 2, 2), 1), ((2, 2, 2), 2), ((2, 2, 1), 3), ((1, 2, 1), 4)]


@pytest.mark.parametrize("n,k", CASES)
def test_poisson_symmetric_constant_kernel_patch_and_energy(n, k):
    dim = len(n)
    lengths = tuple(1.0 + 0.5 * d for d in range(dim))
    lv = box_level(n, lengths, alpha=0.25, seed=7)
    A, pts, node_of, nn = _assemble(lv, k)
    Ad = A.toarray()
    np.testing.assert_allclose(Ad, Ad.T, atol=1e-13 * abs(Ad).max())
    np.testing.assert_allclose(A @ np.ones(nn), 0.0, atol=1e-12 * abs(Ad).max())
    a = np.array([0.7, -1.3, 0.4][:dim])
    u = pts @ a + 0.3
    r = A @ u
    on_bdry = np.zeros(nn, bool)
    for d in range(dim):
        on_bdry |= (np.abs(pts[:, d]) < 1e-12) | (np.abs(pts[:, d] - lengths[d]) < 1e-12)
    np.testing.assert_allclose(r[~on_bdry], 0.0, atol=1e-11 * abs(Ad).max())
    # energy of a linear field: |a|^2 |Omega|
    np.testing.assert_allclose(u @ r, (a @ a) * np.prod(lengths), rtol=1e-12)


@pytest.mark.parametrize("k", [1, 2])
def test_elasticity_rigid_body_modes_and_linear_energy(k):
    lam, mu = 10.0, 1.0
    lv = box_level((4, 2, 2), (4.0, 1.0, 1.0), alpha=0.2, seed=9)
    A, pts, node_of, nn = _assemble(lv, k, 3, (lam, mu))
    Ad = A.toarray()
    np.testing.assert_allclose(Ad, Ad.T, atol=1e-12 * abs(Ad).max())
    x, y, z = pts.T
    one, zero = np.ones(nn), np.zeros(nn)
    modes = [(one, zero, zero), (zero, one, zero), (zero, zero, one),
             (zero, z, -y), (-z, zero, x), (y, -x, zero)]          # Eq. rbm
    for m in modes:
        u = np.stack(m, axis=1).ravel()
        np.testing.assert_allclose(A @ u, 0.0, atol=1e-11 * abs(Ad).max())
    M = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.6], [0.7, 0.2, -0.1]])
    u = (pts @ M.T).ravel()
    eps = 0.5 * (M + M.T)
    energy = 4.0 * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
    np.testing.assert_allclose(u @ (A @ u), energy, rtol=1e-12)


@pytest.mark.parametrize("n,k,ncomp", [((3, 4), 3, 1), ((2, 2, 2), 3, 1), ((2, 1, 2), 2, 3)])
def test_renumbering_and_reorientation_invariance(n, k, ncomp):
    lv = box_level(n, alpha=0.2, seed=3)
    lv2 = scramble(lv, seed=8)
    A1, p1, _, nn = _assemble(lv, k, ncomp, (2.0, 0.5))
    A2, p2, _, _ = _assemble(lv2, k, ncomp, (2.0, 0.5))
    d = np.linalg.norm(p1[:, None] - p2[None], axis=2)
    perm = d.argmin(1)                                   # node i of mesh 1 is node perm[i] of mesh 2
    assert np.all(d[np.arange(nn), perm] < 1e-13)
    idx = (perm[:, None] * ncomp + np.arange(ncomp)).ravel()
    B = A2.toarray()[np.ix_(idx, idx)]
    np.testing.assert_allclose(A1.toarray(), B, atol=1e-12 * abs(B).max())


def test_load_vector_integrates_constants():
    for n, k, ncomp in [((3, 2), 2, 1), ((2, 2, 2), 3, 1), ((3, 1, 1), 2, 3)]:
        lv = box_level(n, tuple(1.0 + d for d in range(len(n))), alpha=0.2, seed=1)
        node_of, nn, _, _ = dofs.number_dofs(lv.cells, k, lv.dim)
        fconst = np.arange(1, ncomp + 1, dtype=float)
        b = assembly.load_vector(lv.vertices, lv.cells, node_of, nn, k, lv.dim,
                                 lambda x: np.tile(fconst, (len(x), 1)), ncomp)
        vol = np.prod([1.0 + d for d in range(len(n))])
        np.testing.assert_allclose(b.reshape(nn, ncomp).sum(0), fconst * vol, rtol=1e-13)


def _l2_error(lv, k, u_nodes, exact):
    from numpy.polynomial import legendre as npleg
    t, w = npleg.leggauss(k + 3)
    mi = fe.multi_indices(k + 3, lv.dim)
    qp = 0.5 * (t[mi] + 1.0)
    qw = np.prod(0.5 * w[mi], axis=1)
    val, _ = fe.tensor_basis(k, lv.dim, qp)
    N, dN = fe.q1_shape(lv.dim, qp)
    X = lv.vertices[lv.cells]
    J = np.einsum("cva,qvb->cqab", X, dN)
    xq = np.einsum("qv,cva->cqa", N, X)
    node_of, _, _, _ = dofs.number_dofs(lv.cells, k, lv.dim)
    uh = np.einsum("qi,ci->cq", val, u_nodes[node_of])
    err = (uh - exact(xq.reshape(-1, lv.dim)).reshape(uh.shape)) ** 2
    return np.sqrt(np.sum(err * np.abs(np.linalg.det(J)) * qw[None]))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_manufactured_solution_converges_at_rate_k_plus_1(k):
    """-Lap u = 2 pi^2 sin(pi x) sin(pi y) on the unit square (config 1's problem)."""
    exact = lambda x: np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])
    f = lambda x: (2 * np.pi ** 2 * exact(x))[:, None]
    errs = []
    ns = [4, 8, 16] if k < 3 else [3, 6, 12]
    for n in ns:
        lv = box_level((n, n), alpha=0.15, seed=n)
        A, pts, node_of, nn = _assemble(lv, k)
        mask = dofs.dirichlet_nodes(lv.cells, lv.dirichlet, node_of, k, 2)
        b = assembly.load_vector(lv.vertices, lv.cells, node_of, nn, k, 2, f)
        fr = np.nonzero(~mask)[0]
        u = np.zeros(nn)
        u[fr] = spla.spsolve(A[fr][:, fr].tocsc(), b[fr])
        errs.append(_l2_error(lv, k, u, exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > k + 1 - 0.35, (errs, rates)
