"""Pins of the oracle's non-nested transfer P and restriction R = P^T (Sec. 2-3)."""
import numpy as np
import pytest

from oracle import dofs, fe, transfer
from tests.oracle_meshes import box_level, scramble


def _level(lv, k):
    node_of, nn, oc, ol = dofs.number_dofs(lv.cells, k, lv.dim)
    mask = dofs.dirichlet_nodes(lv.cells, lv.dirichlet, node_of, k, lv.dim)
    pts = dofs.support_points(lv.vertices, lv.cells, oc, ol, k, lv.dim)
    return dict(vertices=lv.vertices, cells=lv.cells, node_of=node_of, free=~mask, pts=pts, n=nn)


def _P(fine, coarse, k, dim):
    free_f = np.nonzero(fine["free"])[0]
    P, cell, xi = transfer.transfer_matrix(fine["pts"], free_f, coarse, k, dim)
    return P, free_f, cell, xi


@pytest.mark.parametrize("dim,nc,nf,k", [(2, 5, 11, 1), (2, 5, 11, 3), (3, 3, 7, 2), (3, 2, 5, 4)])
def test_reproduces_linear_fields_on_jittered_non_nested_meshes(dim, nc, nf, k):
    c = _level(box_level((nc,) * dim, alpha=0.2, seed=1, dirichlet="none"), k)
    f = _level(box_level((nf,) * dim, alpha=0.2, seed=2, dirichlet="none"), k)
    P, free_f, _, _ = _P(f, c, k, dim)
    a = np.array([0.4, -0.9, 1.3][:dim])
    u = lambda x: x @ a - 0.2
    np.testing.assert_allclose(P @ u(c["pts"]), u(f["pts"][free_f]), atol=1e-13)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 2), (3, 3)])
def test_reproduces_degree_k_polynomials_on_affine_non_nested_meshes(dim, k):
    c = _level(box_level((3,) * dim, dirichlet="none"), k)
    f = _level(box_level((7,) * dim, dirichlet="none"), k)
    P, free_f, _, _ = _P(f, c, k, dim)
    rng = np.random.default_rng(k)
    for _ in range(4):
        e = rng.multinomial(k, [1.0 / (dim + 1)] * (dim + 1))[:dim]   # total degree <= k
        u = lambda x: np.prod(x ** e, axis=1)
        np.testing.assert_allclose(P @ u(c["pts"]), u(f["pts"][free_f]), atol=1e-12)


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 3)])
def test_identical_meshes_give_identity(dim, k):
    lv = box_level((3,) * dim, alpha=0.2, seed=4)
    c = _level(lv, k)
    f = _level(scramble(lv, seed=6), k)        # same geometry, other numbering/orientation
    P, free_f, _, _ = _P(f, c, k, dim)
    Pd = P.toarray()
    Pd[np.abs(Pd) < 1e-12] = 0.0
    assert np.all((Pd == 0) | (np.abs(Pd - 1) < 1e-12))
    assert np.all((Pd != 0).sum(1) == 1) and np.all((Pd != 0).sum(0) == 1)
    # the 1 sits at the coarse node with the same support point
    cols = np.nonzero(c["free"])[0][Pd.argmax(1)]
    np.testing.assert_allclose(c["pts"][cols], f["pts"][free_f], atol=1e-13)


@pytest.mark.parametrize("dim,k", [(2, 3), (3, 2)])
def test_nested_meshes_give_canonical_injection(dim, k):
    """On nested meshes P is the embedding V_{l-1} in V_l (Sec. 4.1): the fine
    interpolant of a coarse function equals it everywhere."""
    c = _level(box_level((2,) * dim, dirichlet="none"), k)
    f = _level(box_level((4,) * dim, dirichlet="none"), k)
    P, free_f, _, _ = _P(f, c, k, dim)
    rng = np.random.default_rng(0)
    uc = rng.standard_normal(c["n"])
    uf = P @ uc
    # evaluate both fields at random points of every fine cell (affine, axis-aligned cells)
    xi = rng.random((9, dim))
    val, _ = fe.tensor_basis(k, dim, xi)
    for cf in range(len(f["cells"])):
        lo = f["vertices"][f["cells"][cf][0]]
        x = lo + xi * 0.25
        fine_vals = val @ uf[f["node_of"][cf]]
        cc = np.floor(x[0] / 0.5).astype(int)
        cidx = int(sum(cc[d] * 2 ** d for d in range(dim)))
        xc = (x - c["vertices"][c["cells"][cidx][0]]) / 0.5
        vc, _ = fe.tensor_basis(k, dim, xc)
        np.testing.assert_allclose(fine_vals, vc @ uc[c["node_of"][cidx]], atol=1e-12)


def test_located_coordinates_map_back_and_lowest_cell_wins():
    c = _level(box_level((4, 4, 3), alpha=0.2, seed=3, dirichlet="none"), 2)
    f = _level(box_level((9, 8, 7), alpha=0.2, seed=8, dirichlet="none"), 2)
    P, free_f, cell, xi = _P(f, c, 2, 3)
    N, _ = fe.q1_shape(3, xi)
    X = c["vertices"][c["cells"][cell]]
    np.testing.assert_allclose(np.einsum("pv,pvd->pd", N, X), f["pts"][free_f], atol=1e-12)
    assert xi.min() >= 0.0 and xi.max() <= 1.0
    # a point on the face shared by coarse cells 0 and 1 (x-neighbours) goes to cell 0
    face_pt = c["vertices"][c["cells"][0][[1, 3, 5, 7]]].mean(0)[None]
    cl, _ = transfer.locate(face_pt, c["vertices"], c["cells"], 3)
    assert cl[0] == 0


def test_nearest_point_fallback_outside_domain():
    c = _level(box_level((3, 3), dirichlet="none"), 1)
    pts = np.array([[1.0 + 1e-3, 0.5], [-2e-3, -1e-3]])
    cell, xi = transfer.locate(pts, c["vertices"], c["cells"], 2)
    assert cell[0] == 5 and abs(xi[0, 0] - 1.0) < 1e-15 and abs(xi[0, 1] - 0.5) < 1e-12
    assert cell[1] == 0 and np.all(xi[1] == 0.0)


def test_restriction_is_transpose():
    c = _level(box_level((3, 3), alpha=0.2, seed=1), 2)
    f = _level(box_level((7, 7), alpha=0.2, seed=2), 2)
    P, _, _, _ = _P(f, c, 2, 2)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(P.shape[1])
    y = rng.standard_normal(P.shape[0])
    assert abs((P @ x) @ y - x @ (P.T @ y)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)


def test_located_points_are_true_preimages_in_distorted_cells():
    """Deformed cube, Q4: in strongly distorted coarse cells Newton can wander
    into [0,1]^3 without converging for points outside the cell; only a
    converged inversion (Sec. 3.1) may be accepted, so every located xi maps
    back to its point."""
    from synthetic import config_levels
    c_lv, f_lv = config_levels("c3_3d_q4_deformed", n_levels=2)
    fn, fnn, oc, ol = dofs.number_dofs(f_lv.cells, 4, 3)
    pts = dofs.support_points(f_lv.vertices, f_lv.cells, oc, ol, 4, 3)
    cell, xi = transfer.locate(pts, c_lv.vertices, c_lv.cells, 3)
    N, _ = fe.q1_shape(3, xi)
    X = c_lv.vertices[c_lv.cells[cell]]
    np.testing.assert_allclose(np.einsum("pv,pvd->pd", N, X), pts, rtol=0, atol=1e-12)
    # the non-converged iterates exist: Newton from the centre of coarse cell 8
    # does not converge for one of these points
    p = pts[np.argmin(np.linalg.norm(pts - np.array([0.26927729, 0.71235964, 0.08251205]), axis=1))]
    _, conv = transfer.newton_inverse(p[None], c_lv.vertices[c_lv.cells[[8]]], 3)
    assert not conv[0]


@pytest.mark.parametrize("dim,kc,kf", [(2, 1, 2), (2, 3, 4), (3, 1, 2), (3, 2, 3)])
def test_degree_change_on_one_mesh_is_the_canonical_embedding(dim, kc, kf):
    """Polynomial coarsening (Sec. 2, "Coarse grid solvers"): on one mesh Q_kc is
    contained in Q_kf, so P interpolates the coarse field exactly at every point."""
    lv = box_level((3,) * dim, alpha=0.2, seed=2, dirichlet="none")
    c = _level(lv, kc)
    f = _level(lv, kf)
    P, free_f, cell, xi = _P(f, c, kc, dim)
    rng = np.random.default_rng(4)
    uc = rng.standard_normal(c["n"])
    uf = P @ uc
    xr = rng.random((7, dim))
    vf, _ = fe.tensor_basis(kf, dim, xr)
    vc, _ = fe.tensor_basis(kc, dim, xr)
    for K in range(len(lv.cells)):
        np.testing.assert_allclose(vf @ uf[f["node_of"][K]], vc @ uc[c["node_of"][K]], atol=1e-12)


@pytest.mark.parametrize("k", [1, 3])
def test_curved_boundary_points_are_projected(k):
    """Annulus levels meshed independently (Sec. 3.3): fine Neumann points on the
    outer circle lie outside the coarse polygon; they are assigned the nearest
    coarse cell with xi projected onto the reference cell.  P keeps the
    partition of unity there, and the projected point is within the gap
    between the polygons (O(h^2))."""
    from synthetic.meshes import annulus_level
    c_lv, f_lv = annulus_level(3, 10, seed=1), annulus_level(7, 23, seed=2)
    c = _level(c_lv, k)
    f = _level(f_lv, k)
    P, free_f, cell, xi = _P(f, c, k, 2)
    pts = f["pts"][free_f]
    # partition of unity where the coarse cell has no Dirichlet (dropped) nodes:
    # the outer ring of the coarse mesh, r > 5/6
    outer = np.linalg.norm(pts, axis=1) > 0.85
    np.testing.assert_allclose((P @ np.ones(P.shape[1]))[outer], 1.0, atol=1e-12)
    N, _ = fe.q1_shape(2, xi)
    mapped = np.einsum("pv,pvd->pd", N, c["vertices"][c["cells"][cell]])
    r = np.linalg.norm(pts, axis=1)
    outside = np.linalg.norm(mapped - pts, axis=1) > 1e-12
    assert outside.sum() > 0 and np.all(r[outside] > 0.9)          # only near the outer circle
    h = 2 * np.pi / 10
    assert np.max(np.linalg.norm(mapped - pts, axis=1)) < h * h
