"""Jittered structured quad/hex meshes for the five benchmark configurations.

Conventions (an input format, not part of the method):
  * vertices: float64 array [n_vertices, dim], lexicographic, x fastest;
  * cells: int32 array [n_cells, 2**dim]; local vertex v = b0 + 2*b1 + 4*b2
    where b_d is the offset bit of that corner in direction d;
  * dirichlet: uint8 array [n_vertices], 1 where a vertex lies on the
    Dirichlet part of the boundary.
Random numbers come from a splitmix64 stream (Steele, Lea, Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), consumed one draw
per coordinate for every vertex in lexicographic order; only interior
vertices are moved.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """Return the first n outputs of the splitmix64 stream started at seed."""
    with np.errstate(over="ignore"):
        gamma = np.uint64(0x9E3779B97F4A7C15)
        state = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
                 + gamma * np.arange(1, n + 1, dtype=np.uint64)) & _MASK
        z = state
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n doubles uniform in [-1, 1) from the top 53 bits of splitmix64."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def structured_grid(n: tuple, lengths: tuple):
    """Vertices and cells of an n[0] x n[1] (x n[2]) box [0,L0]x[0,L1](x[0,L2])."""
    dim = len(n)
    axes = [np.linspace(0.0, float(lengths[d]), n[d] + 1) for d in range(dim)]
    grids = np.meshgrid(*axes, indexing="ij")
    # lexicographic, x fastest: flatten in Fortran order of (x, y, z) indices
    verts = np.stack([g.ravel(order="F") for g in grids], axis=1)
    nv = [n[d] + 1 for d in range(dim)]
    idx = np.arange(int(np.prod(nv))).reshape(nv, order="F")
    cidx = [np.arange(n[d]) for d in range(dim)]
    cg = np.meshgrid(*cidx, indexing="ij")
    base = [g.ravel(order="F") for g in cg]
    corners = []
    for v in range(2 ** dim):
        off = [(v >> d) & 1 for d in range(dim)]
        corners.append(idx[tuple(base[d] + off[d] for d in range(dim))])
    cells = np.stack(corners, axis=1).astype(np.int32)
    return verts, cells


def boundary_vertex_mask(verts: np.ndarray, lengths: tuple) -> np.ndarray:
    on = np.zeros(len(verts), dtype=bool)
    for d in range(verts.shape[1]):
        on |= (verts[:, d] == 0.0) | (verts[:, d] == float(lengths[d]))
    return on


def jitter_interior(verts, n, lengths, alpha, seed):
    """Move interior vertices by U(-alpha*h_d, alpha*h_d) per coordinate."""
    dim = verts.shape[1]
    h = np.array([lengths[d] / n[d] for d in range(dim)])
    draws = uniform_pm1(seed, verts.size).reshape(verts.shape)
    moved = verts + alpha * h[None, :] * draws
    interior = ~boundary_vertex_mask(verts, lengths)
    out = verts.copy()
    out[interior] = moved[interior]
    return out


def deform_sine(verts, amp=0.08):
    """x -> x + amp*sin(2 pi x) sin(2 pi y) sin(2 pi z), added to every component."""
    s = np.prod(np.sin(2.0 * np.pi * verts), axis=1)
    return verts + amp * s[:, None]


@dataclass
class Level:
    dim: int
    vertices: np.ndarray
    cells: np.ndarray
    dirichlet: np.ndarray
    n: tuple = field(default=())


def _level(n, lengths, alpha, seed, dirichlet="all", deform=False):
    verts, cells = structured_grid(n, lengths)
    if alpha > 0:
        verts = jitter_interior(verts, n, lengths, alpha, seed)
    if deform:
        verts = deform_sine(verts)
    if dirichlet == "all":
        dmask = boundary_vertex_mask(structured_grid(n, lengths)[0], lengths)
    elif dirichlet == "x0":
        dmask = structured_grid(n, lengths)[0][:, 0] == 0.0
    else:
        raise ValueError(dirichlet)
    return Level(len(n), np.ascontiguousarray(verts, dtype=np.float64),
                 np.ascontiguousarray(cells, dtype=np.int32),
                 dmask.astype(np.uint8), tuple(n))


# The benchmark configurations.  Cell counts per level, coarse -> fine.
CONFIGS = {
    "c1_2d_q1": dict(dim=2, degree=1, ncomp=1, cheb=3, nrhs=1,
                     cells=[(5, 5), (11, 11), (23, 23)], lengths=(1.0, 1.0),
                     alpha=0.2, seeds="stream0", dirichlet="all", deform=False),
    "c2_3d_q2": dict(dim=3, degree=2, ncomp=1, cheb=3, nrhs=8,
                     cells=[(6,) * 3, (13,) * 3, (27,) * 3, (55,) * 3],
                     lengths=(1.0, 1.0, 1.0), alpha=0.15, seeds=[1, 2, 3, 4],
                     dirichlet="all", deform=False),
    "c3_3d_q4_deformed": dict(dim=3, degree=4, ncomp=1, cheb=5, nrhs=4,
                              cells=[(4,) * 3, (9,) * 3, (19,) * 3, (39,) * 3],
                              lengths=(1.0, 1.0, 1.0), alpha=0.1,
                              seeds=[101, 102, 103, 104], dirichlet="all",
                              deform=True),
    "c4_3d_q2_elasticity": dict(dim=3, degree=2, ncomp=3, cheb=4, nrhs=1,
                                cells=[(8, 2, 2), (19, 5, 5), (41, 11, 11)],
                                lengths=(4.0, 1.0, 1.0), alpha=0.1,
                                seeds=[201, 202, 203], dirichlet="x0",
                                deform=False, lame=(10.0, 1.0)),
}


def config_levels(name: str, n_levels: int | None = None, cells=None):
    """Levels (coarse -> fine) of a named configuration.

    n_levels keeps only the coarsest n_levels levels; cells overrides the
    per-level cell counts (used for small test variants of a family).
    """
    cfg = CONFIGS[name]
    cl = list(cells if cells is not None else cfg["cells"])
    if n_levels is not None:
        cl = cl[:n_levels]
    levels = []
    if cfg["seeds"] == "stream0":
        # one stream seeded 0, consumed level by level from coarse to fine
        offset = 0
        for n in cl:
            verts, cells_ = structured_grid(n, cfg["lengths"])
            draws = uniform_pm1(0, offset + verts.size)[offset:].reshape(verts.shape)
            offset += verts.size
            h = np.array([cfg["lengths"][d] / n[d] for d in range(cfg["dim"])])
            interior = ~boundary_vertex_mask(verts, cfg["lengths"])
            v2 = verts.copy()
            v2[interior] = (verts + cfg["alpha"] * h[None, :] * draws)[interior]
            dmask = boundary_vertex_mask(verts, cfg["lengths"])
            levels.append(Level(cfg["dim"], v2, cells_, dmask.astype(np.uint8), tuple(n)))
    else:
        seeds = list(cfg["seeds"])
        for i, n in enumerate(cl):
            seed = seeds[i] if i < len(seeds) else seeds[-1] + (i - len(seeds) + 1)
            levels.append(_level(n, cfg["lengths"], cfg["alpha"], seed,
                                 cfg["dirichlet"], cfg["deform"]))
    return levels


def family_levels(dim, cells_fine, n_levels, alpha, seed, lengths=None,
                  dirichlet="all", ratio=2.2):
    """A jittered family: fine level n, coarser n_{l-1} = floor((n_l - 1)/ratio)."""
    lengths = lengths or (1.0,) * dim
    ns = [cells_fine]
    while len(ns) < n_levels:
        ns.append(max(1, int((ns[-1] - 1) // ratio)))
    ns = ns[::-1]
    return [_level((n,) * dim, lengths, alpha, seed + i, dirichlet) for i, n in enumerate(ns)]


def annulus_level(n_r, n_t, r0=0.5, r1=1.0, alpha=0.1, seed=0, n_z=0, height=1.0):
    """Quad (n_z = 0) or hex mesh of the annulus r0 <= r <= r1 (times [0, height]).

    Vertices on the circles r = r0 and r = r1 lie exactly on them; the cells are
    Q1, so each level's boundary is a different polygon inscribed in the
    circles: fine boundary points fall outside coarser levels.  Interior
    vertices are jittered in (r, theta) by +-alpha of the spacing (splitmix64,
    one draw per coordinate per vertex).  Dirichlet flags mark r = r0.
    """
    nr1 = n_r + 1
    r = np.linspace(r0, r1, nr1)
    t = np.linspace(0.0, 2 * np.pi, n_t + 1)[:-1]
    nz1 = n_z + 1 if n_z else 1
    z = np.linspace(0.0, height, nz1) if n_z else np.zeros(1)
    R, T, Z = np.meshgrid(r, t, z, indexing="ij")
    R, T, Z = (a.ravel(order="F") for a in (R, T, Z))
    draws = uniform_pm1(seed, 3 * R.size).reshape(R.size, 3)
    interior_r = (R > r0) & (R < r1)
    R = np.where(interior_r, R + alpha * (r1 - r0) / n_r * draws[:, 0], R)
    T = T + alpha * (2 * np.pi / n_t) * draws[:, 1]
    if n_z:
        iz = (Z > 0) & (Z < height)
        Z = np.where(iz, Z + alpha * height / n_z * draws[:, 2], Z)
    idx = np.arange(R.size).reshape((nr1, n_t, nz1), order="F")
    cells = []
    for k in range(max(n_z, 1)):
        for j in range(n_t):
            for i in range(n_r):
                jp = (j + 1) % n_t
                c = [idx[i, j, k], idx[i + 1, j, k], idx[i, jp, k], idx[i + 1, jp, k]]
                if n_z:
                    c += [idx[i, j, k + 1], idx[i + 1, j, k + 1], idx[i, jp, k + 1], idx[i + 1, jp, k + 1]]
                cells.append(c)
    cells = np.array(cells, dtype=np.int32)
    xy = np.stack([R * np.cos(T), R * np.sin(T)] + ([Z] if n_z else []), axis=1)
    dirichlet = (np.abs(R - r0) < 1e-14).astype(np.uint8)
    dim = 3 if n_z else 2
    return Level(dim, np.ascontiguousarray(xy), cells, dirichlet, (n_r, n_t) + ((n_z,) if n_z else ()))


def refine_nested(level: Level):
    """Uniform refinement of a structured level (from structured_grid, possibly
    jittered): every cell is split into 2^d children by mapping the reference
    midpoints through the cell's Q1 map, so the refined space contains the
    coarse one.  Returns (fine Level, parent cell [n_fine_cells] int32,
    child index [n_fine_cells] uint8 with bit d = position in direction d)."""
    n = level.n
    dim = len(n)
    nf = tuple(2 * m for m in n)
    nv_c = [m + 1 for m in n]
    nv_f = [m + 1 for m in nf]
    vf = np.empty((int(np.prod(nv_f)), dim))
    grids = np.meshgrid(*[np.arange(m) for m in nv_f], indexing="ij")
    I = [g.ravel(order="F") for g in grids]                       # fine vertex multi-index
    cidx = [np.minimum(I[d] // 2, n[d] - 1) for d in range(dim)]   # a coarse cell containing it
    eta = [(I[d] - 2 * cidx[d]) / 2.0 for d in range(dim)]         # 0, 1/2 or 1
    cell = sum(cidx[d] * int(np.prod(n[:d])) for d in range(dim))
    X = level.vertices[level.cells[cell]]                          # [nv, 2^d, dim]
    w = np.ones((len(cell), 2 ** dim))
    for v in range(2 ** dim):
        for d in range(dim):
            w[:, v] *= eta[d] if (v >> d) & 1 else 1.0 - eta[d]
    vf[:] = np.einsum("pv,pvd->pd", w, X)
    _, cells_f = structured_grid(nf, (1.0,) * dim)
    cg = np.meshgrid(*[np.arange(m) for m in nf], indexing="ij")
    J = [g.ravel(order="F") for g in cg]
    parent = sum((J[d] // 2) * int(np.prod(n[:d])) for d in range(dim)).astype(np.int32)
    child = sum((J[d] % 2) << d for d in range(dim)).astype(np.uint8)
    dmask = np.zeros(len(vf), dtype=np.uint8)
    on = np.zeros(len(vf), dtype=bool)
    for d in range(dim):
        on |= (I[d] == 0) | (I[d] == nv_f[d] - 1)
    # a fine boundary vertex is Dirichlet if its coarse boundary face is
    if level.dirichlet.any():
        dmask[on] = 1
    return Level(dim, vf, cells_f.astype(np.int32), dmask, nf), parent, child
