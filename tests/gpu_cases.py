"""Shared builders for the GPU parity tests: the same seeded levels go to the
oracle and to the CUDA library."""
import functools

import numpy as np

from synthetic import config_levels
from synthetic.meshes import CONFIGS, annulus_level
from tests.oracle_meshes import box_level, scramble

# name -> (levels factory, degree, ncomp, lame, cheb, nrhs)
CASES = {
    "c1_q1": (lambda: config_levels("c1_2d_q1"), 1, 1, (1.0, 1.0), 3, 1),
    "c1_q3": (lambda: config_levels("c1_2d_q1", n_levels=2), 3, 1, (1.0, 1.0), 3, 3),
    "c1_q2_16rhs": (lambda: config_levels("c1_2d_q1"), 2, 1, (1.0, 1.0), 3, 16),
    "c1_q4_5rhs": (lambda: config_levels("c1_2d_q1", n_levels=2), 4, 1, (1.0, 1.0), 3, 5),
    "c2_q1_3lev": (lambda: config_levels("c2_3d_q2", n_levels=3), 1, 1, (1.0, 1.0), 3, 2),
    "c2_q2_3lev": (lambda: config_levels("c2_3d_q2", n_levels=3), 2, 1, (1.0, 1.0), 3, 8),
    "c3_q4_2lev": (lambda: config_levels("c3_3d_q4_deformed", n_levels=2), 4, 1, (1.0, 1.0), 5, 4),
    "c4_elast": (lambda: config_levels("c4_3d_q2_elasticity"), 2, 3, (10.0, 1.0), 4, 1),
    # the largest channel count: 3 components x 16 right-hand sides
    "c4_elast_16rhs": (lambda: config_levels("c4_3d_q2_elasticity", n_levels=2), 2, 3, (10.0, 1.0),
                       4, 16),
    "scrambled_q3": (lambda: [scramble(box_level((2, 2, 2), alpha=0.1, seed=3), 5),
                              scramble(box_level((5, 4, 3), alpha=0.2, seed=4), 6)], 3, 1,
                     (1.0, 1.0), 3, 2),
    # curved domains with a Neumann outer boundary (Sec. 3.3): fine points outside
    # the coarser polygonal boundaries go through the nearest-point projection
    "annulus_q2": (lambda: [annulus_level(2, 12, seed=1), annulus_level(5, 27, seed=2),
                            annulus_level(11, 57, seed=3)], 2, 1, (1.0, 1.0), 3, 2),
    "cylinder_q2": (lambda: [annulus_level(2, 8, n_z=2, seed=4), annulus_level(4, 17, n_z=4, seed=5)],
                    2, 1, (1.0, 1.0), 3, 1),
    # polynomial coarsening on the coarsest mesh below the non-nested levels
    "c3_q4_pmg": (lambda: [config_levels("c3_3d_q4_deformed", n_levels=1)[0]] * 4
                  + config_levels("c3_3d_q4_deformed", n_levels=2)[1:], 4, 1, (1.0, 1.0), 5, 4,
                  [1, 2, 3, 4, 4]),
}


def degrees(name):
    c = CASES[name]
    return c[6] if len(c) > 6 else None


@functools.lru_cache(maxsize=None)
def oracle_case(name):
    from oracle.hierarchy import OracleHierarchy
    lv, k, nc, lame, cheb, nrhs = CASES[name][:6]
    levels = lv()
    return levels, OracleHierarchy(levels, k, nc, lame, cheb, level_degrees=degrees(name))


def gpu_case(name, levels, **kw):
    from paper_2412_10910_gb300 import nnmg
    _, k, nc, lame, cheb, nrhs = CASES[name][:6]
    return nnmg.Hierarchy(levels, k, nc, lame, cheb, max_nrhs=16, level_degrees=degrees(name), **kw)


def rng_vec(rows, nrhs, seed):
    return np.random.default_rng(seed).standard_normal((rows, nrhs))
