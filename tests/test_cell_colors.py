"""Host-side cell coloring of the deterministic mode (nnmg_color_cells, no
GPU): no two cells of one color share a vertex, the colors are the greedy
ones (each cell takes the smallest color that no earlier cell sharing a
vertex took), structured grids in lexicographic order need 2^d colors, and
bad input is rejected."""
import numpy as np
import pytest

from paper_2412_10910_gb300 import _abi, nnmg
from synthetic.meshes import annulus_level, structured_grid
from tests.oracle_meshes import box_level, scramble


def _neighbors(cells):
    by_vertex = {}
    for c, vs in enumerate(cells):
        for v in vs:
            by_vertex.setdefault(int(v), set()).add(c)
    return [set().union(*(by_vertex[int(v)] for v in vs)) - {c} for c, vs in enumerate(cells)]


def _check_greedy(cells, color, n):
    nb = _neighbors(cells)
    assert color.max() + 1 == n
    for c in range(len(cells)):
        assert all(color[d] != color[c] for d in nb[c])                  # a valid coloring
        earlier = {int(color[d]) for d in nb[c] if d < c}
        assert color[c] == min(set(range(65)) - earlier)                  # the greedy choice


@pytest.mark.parametrize("n", [(5, 4), (3, 4, 2), (6, 5, 4)])
def test_structured_grids_take_two_to_the_d_colors(n):
    verts, cells = structured_grid(n, (1.0,) * len(n))
    color, k = nnmg.nnmg_color_cells(cells, len(verts))
    assert k == 2 ** len(n)
    _check_greedy(cells, color, k)


@pytest.mark.parametrize("mesh", ["scrambled", "annulus", "cylinder"])
def test_unstructured_orders_give_valid_greedy_colorings(mesh):
    if mesh == "scrambled":
        lv = scramble(box_level((5, 4, 3), alpha=0.2, seed=4), 6)
    elif mesh == "annulus":
        lv = annulus_level(4, 24, seed=2)
    else:
        lv = annulus_level(3, 16, n_z=3, seed=5)
    color, k = nnmg.nnmg_color_cells(lv.cells, len(lv.vertices))
    _check_greedy(np.asarray(lv.cells), color, k)


def test_bad_input_is_rejected():
    verts, cells = structured_grid((2, 2), (1.0, 1.0))
    bad = cells.copy()
    bad[0, 0] = len(verts)
    with pytest.raises(nnmg.NNMGError) as e:
        nnmg.nnmg_color_cells(bad, len(verts))
    assert e.value.status == _abi.INVALID_ARG
    # 65 quadrilaterals around one vertex: the last needs a 66th color
    star = np.array([[0, 1 + 3 * i, 2 + 3 * i, 3 + 3 * i] for i in range(66)], dtype=np.int32)
    with pytest.raises(nnmg.NNMGError) as e:
        nnmg.nnmg_color_cells(star, int(star.max()) + 1)
    assert e.value.status == _abi.BAD_MESH
