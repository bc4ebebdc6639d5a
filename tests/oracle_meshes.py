"""Small mesh helpers for the oracle tests (inputs only: topology and coordinates)."""
import itertools

import numpy as np

from synthetic.meshes import Level, structured_grid, boundary_vertex_mask, jitter_interior


def box_level(n, lengths=None, alpha=0.0, seed=0, dirichlet="all", shift=0.0):
    dim = len(n)
    lengths = lengths or (1.0,) * dim
    v, c = structured_grid(n, lengths)
    mask = boundary_vertex_mask(v, lengths)
    if alpha:
        v = jitter_interior(v, n, lengths, alpha, seed)
    if dirichlet == "none":
        mask[:] = False
    return Level(dim, v + shift, c, mask.astype(np.uint8), tuple(n))


def proper_symmetries(dim):
    """(axis permutation, flips) of the reference cell with determinant +1."""
    out = []
    for perm in itertools.permutations(range(dim)):
        sgn = np.linalg.det(np.eye(dim)[list(perm)])
        for flips in itertools.product((0, 1), repeat=dim):
            if sgn * (-1) ** sum(flips) > 0:
                out.append((perm, flips))
    return out


def scramble(level, seed):
    """Permute vertex ids and re-orient every cell by a random proper symmetry."""
    rng = np.random.default_rng(seed)
    dim = level.dim
    nv = len(level.vertices)
    perm_v = rng.permutation(nv)                     # new id of old vertex
    inv = np.argsort(perm_v)
    verts = level.vertices[inv]
    dmask = level.dirichlet[inv]
    syms = proper_symmetries(dim)
    cells = np.empty_like(level.cells)
    for c in range(len(level.cells)):
        axes, flips = syms[rng.integers(len(syms))]
        for vnew in range(2 ** dim):
            bits_new = [(vnew >> d) & 1 for d in range(dim)]
            bits_old = [0] * dim
            for d in range(dim):
                bits_old[axes[d]] = bits_new[d] ^ flips[d]
            vold = sum(b << d for d, b in enumerate(bits_old))
            cells[c, vnew] = perm_v[level.cells[c, vold]]
    cells = cells[rng.permutation(len(cells))]
    return Level(dim, verts, cells, dmask, level.n)
