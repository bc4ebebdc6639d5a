"""The synthetic levels of the benchmark configurations have the sizes the
configurations state: cell counts per level, and DoF counts (all nodes and
free nodes) from the oracle's numbering on the smaller levels and from the
structured closed forms (k n_d + 1 nodes per direction; k n_d - 1 free ones
with a fully Dirichlet boundary) on the large ones."""
import numpy as np
import pytest

from oracle import dofs
from synthetic import config_levels
from synthetic.meshes import CONFIGS

# name: (cells per level, fine nodes x components, fine free DoFs, coarsest free DoFs)
EXPECT = {
    "c1_2d_q1": ([(5, 5), (11, 11), (23, 23)], 576, 484, 16),
    "c2_3d_q2": ([(6,) * 3, (13,) * 3, (27,) * 3, (55,) * 3], 1_367_631, 1_295_029, 1331),
    "c3_3d_q4_deformed": ([(4,) * 3, (9,) * 3, (19,) * 3, (39,) * 3], 3_869_893, 3_723_875, 3375),
    "c4_3d_q2_elasticity": ([(8, 2, 2), (19, 5, 5), (41, 11, 11)], 131_721, 130_134, 1200),
}


def _counts(lv, k, dim):
    node_of, nn, _, _ = dofs.number_dofs(lv.cells, k, dim)
    cons = dofs.dirichlet_nodes(lv.cells, lv.dirichlet, node_of, k, dim)
    return nn, nn - int(cons.sum())


@pytest.mark.parametrize("name", sorted(EXPECT))
def test_config_level_sizes(name):
    cells, fine_all, fine_free, coarse_free = EXPECT[name]
    cfg = CONFIGS[name]
    k, dim, nc = cfg["degree"], cfg["dim"], cfg["ncomp"]
    levels = config_levels(name)
    assert [tuple(lv.n) for lv in levels] == cells
    for lv in levels:
        assert len(lv.cells) == np.prod(lv.n)
    nn0, free0 = _counts(levels[0], k, dim)
    assert free0 * nc == coarse_free
    fine = levels[-1]
    if np.prod(fine.n) <= 50_000:
        nn, free = _counts(fine, k, dim)
    else:
        nn = int(np.prod([k * m + 1 for m in fine.n]))
        free = int(np.prod([k * m - 1 for m in fine.n]))
        # the closed form holds on the numbered levels below
        for lv in levels[:-1]:
            if np.prod(lv.n) <= 20_000:
                assert _counts(lv, k, dim) == (int(np.prod([k * m + 1 for m in lv.n])),
                                               int(np.prod([k * m - 1 for m in lv.n])))
    assert nn * nc == fine_all and free * nc == fine_free
