"""Pins of the oracle's DoF numbering, Dirichlet set and support points."""
import os

import numpy as np
import pytest

from oracle import dofs, fe
from tests.oracle_meshes import box_level, scramble

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nested_dof_counts.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            rows.append(tuple(int(t) for t in line.split()))
    return rows


@pytest.mark.parametrize("dim,p,l,expect", _golden_rows())
def test_dof_counts_match_paper_nested_tables(dim, p, l, expect):
    lv = box_level((2 ** (l - 1),) * dim, (2.0,) * dim, shift=-1.0)
    _, n, _, _ = dofs.number_dofs(lv.cells, p, dim)
    assert n == expect


@pytest.mark.parametrize("n,k", [((3, 4), 1), ((3, 4), 4), ((2, 3, 2), 2), ((2, 2, 3), 3), ((2, 2, 2), 4)])
def test_support_points_consistent_and_distinct(n, k):
    dim = len(n)
    lv = scramble(box_level(n, alpha=0.2, seed=5), seed=11)
    node_of, nn, oc, ol = dofs.number_dofs(lv.cells, k, dim)
    pts = dofs.support_points(lv.vertices, lv.cells, oc, ol, k, dim)
    # every (cell, local node) maps to the point of its global node
    xi = fe.gauss_lobatto_nodes(k)[fe.multi_indices(k + 1, dim)]
    N, _ = fe.q1_shape(dim, xi)
    X = lv.vertices[lv.cells]
    allpts = np.einsum("iv,cvd->cid", N, X)
    np.testing.assert_allclose(allpts, pts[node_of], atol=1e-14)
    # distinct nodes have distinct points, count equals the structured count
    assert nn == np.prod([k * m + 1 for m in n])
    d = np.linalg.norm(pts[:, None] - pts[None], axis=2) + np.eye(nn)
    assert d.min() > 1e-3


def test_first_touch_order():
    lv = box_level((2, 1))
    node_of, nn, oc, ol = dofs.number_dofs(lv.cells, 2, 2)
    assert list(node_of[0]) == list(range(9))
    assert oc[9] == 1 and ol[9] == 1               # first new node of cell 1 is its local node 1
    assert node_of[1][0] == node_of[0][2]          # shared edge, bottom corner


@pytest.mark.parametrize("n,k", [((4, 5), 1), ((4, 5), 3), ((3, 2, 2), 2), ((2, 2, 2), 4)])
def test_dirichlet_count_full_boundary(n, k):
    dim = len(n)
    lv = scramble(box_level(n, alpha=0.1, seed=2), seed=4)
    node_of, nn, _, _ = dofs.number_dofs(lv.cells, k, dim)
    mask = dofs.dirichlet_nodes(lv.cells, lv.dirichlet, node_of, k, dim)
    assert nn - mask.sum() == np.prod([k * m - 1 for m in n])


def test_dirichlet_one_face_only():
    from synthetic.meshes import config_levels
    lv = config_levels("c4_3d_q2_elasticity")[0]       # 8x2x2 beam clamped at x = 0
    node_of, nn, oc, ol = dofs.number_dofs(lv.cells, 2, 3)
    mask = dofs.dirichlet_nodes(lv.cells, lv.dirichlet, node_of, 2, 3)
    pts = dofs.support_points(lv.vertices, lv.cells, oc, ol, 2, 3)
    assert mask.sum() == 5 * 5
    np.testing.assert_array_equal(mask, np.abs(pts[:, 0]) < 1e-14)
