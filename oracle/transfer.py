"""Non-nested transfer by point location (Sec. 2 Eqs. pointwise..residual2, Sec. 3.1, Sec. 3.3).

P[i, j] = phi^{l-1}_j(x_i): the coarse basis function j evaluated at the
support point x_i of fine DoF i.  To evaluate it the oracle finds, for every
fine point, a coarse cell K containing it and the reference coordinates
xi = F_K^{-1}(x_i) by Newton's method on the Q1 map (Sec. 3.1).

Brute force: every coarse cell is a candidate, in index order.  A cell whose
bounding box (widened by 1e-9 of the domain size) misses the point cannot
contain it, so it is skipped without changing the result.  Newton starts at
xi = (1/2, ...), runs at most 30 steps and stops once max|dxi| < 1e-14; it has
inverted the map only if its last step was below 1e-10 (in a strongly
distorted cell the iterates of a point outside it can wander into [0,1]^d
without converging, and such an iterate is not a preimage).  A cell accepts
the point when Newton converged and xi lies in [-1e-10, 1 + 1e-10]^d; the
first accepting cell wins.  If no cell accepts, the converged cell whose xi is
nearest to [0,1]^d is taken (lowest index on ties) and xi is projected onto
[0,1]^d (Eq. closest_point).
Restriction is R = P^T (Eq. residual2).
"""
import numpy as np
import scipy.sparse as sp

from .fe import q1_shape, tensor_basis

ACCEPT_TOL = 1e-10
NEWTON_MAXIT = 30
NEWTON_STOP = 1e-14
NEWTON_CONVERGED = 1e-10


def newton_inverse(points, X, dim):
    """(xi, converged): Newton for F(xi) = points, Q1 maps with corners X [P, nv, dim].

    xi is NaN after a singular Jacobian; converged is False unless the last
    Newton step was below NEWTON_CONVERGED.
    """
    P = points.shape[0]
    xi = np.full((P, dim), 0.5)
    last = np.full(P, np.inf)
    active = np.ones(P, dtype=bool)
    for _ in range(NEWTON_MAXIT):
        if not active.any():
            break
        a = np.nonzero(active)[0]
        N, dN = q1_shape(dim, xi[a])
        F = np.einsum("pv,pvd->pd", N, X[a])
        J = np.einsum("pvd,pvb->pdb", X[a], dN)
        with np.errstate(all="ignore"):
            det = np.linalg.det(J)
            ok = np.isfinite(det) & (det != 0)
            dx = np.full((len(a), dim), np.nan)
            if ok.any():
                dx[ok] = np.linalg.solve(J[ok], (F - points[a])[ok][..., None])[..., 0]
        xi[a] = xi[a] - dx
        step = np.max(np.abs(dx), axis=1)
        last[a] = step
        done = ~(step >= NEWTON_STOP)                           # converged or NaN
        active[a[done]] = False
    return xi, last < NEWTON_CONVERGED


def _dist_to_unit(xi, converged):
    clamped = np.clip(xi, 0.0, 1.0)
    d = np.sqrt(np.sum((xi - clamped) ** 2, axis=1))
    return np.where(np.isfinite(d) & converged, d, np.inf)


def locate(points, coarse_vertices, coarse_cells, dim, chunk=2048):
    """(cell [P], xi [P, dim]) for every point, clamped to [0,1]^d."""
    X = coarse_vertices[coarse_cells]                       # [nc, nv, dim]
    span = coarse_vertices.max(0) - coarse_vertices.min(0)
    eps = 1e-9 * float(np.max(span))
    lo = X.min(axis=1) - eps
    hi = X.max(axis=1) + eps
    P = points.shape[0]
    cell = np.full(P, -1, dtype=np.int64)
    xi = np.zeros((P, dim))
    for p0 in range(0, P, chunk):
        pts = points[p0:p0 + chunk]
        inside = np.all((pts[:, None, :] >= lo[None]) & (pts[:, None, :] <= hi[None]), axis=2)
        pi, ci = np.nonzero(inside)                         # row-major: cells ascending per point
        if len(pi):
            x, conv = newton_inverse(pts[pi], X[ci], dim)
            ok = conv & np.all((x >= -ACCEPT_TOL) & (x <= 1.0 + ACCEPT_TOL), axis=1)
            sel = np.nonzero(ok)[0]
            if len(sel):
                up, first = np.unique(pi[sel], return_index=True)
                cell[p0 + up] = ci[sel[first]]
                xi[p0 + up] = x[sel[first]]
    # nearest-point fallback (Sec. 3.3): search all cells
    for p in np.nonzero(cell < 0)[0]:
        x, conv = newton_inverse(np.repeat(points[p][None], len(X), 0), X, dim)
        d = _dist_to_unit(x, conv)
        c = int(np.argmin(d))
        if not np.isfinite(d[c]):
            raise RuntimeError("point not found")
        cell[p], xi[p] = c, x[c]
    return cell, np.clip(xi, 0.0, 1.0)


def transfer_matrix(fine_points, fine_free_nodes, coarse, k, dim):
    """Node-level P over free DoFs: rows = free fine nodes, cols = free coarse nodes.

    `coarse` is a dict with vertices, cells, node_of, free (bool mask over nodes).
    Returns (P csr [n_free_f, n_free_c], cell, xi) for the located points.
    """
    pts = fine_points[fine_free_nodes]
    cell, xi = locate(pts, coarse["vertices"], coarse["cells"], dim)
    val, _ = tensor_basis(k, dim, xi)                       # [P, nloc]
    cnodes = coarse["node_of"][cell]                        # [P, nloc]
    col_of = -np.ones(len(coarse["free"]), dtype=np.int64)
    col_of[coarse["free"]] = np.arange(int(coarse["free"].sum()))
    cols = col_of[cnodes]
    rows = np.repeat(np.arange(len(pts))[:, None], cnodes.shape[1], axis=1)
    keep = cols >= 0
    P = sp.csr_matrix((val[keep], (rows[keep], cols[keep])),
                      shape=(len(pts), int(coarse["free"].sum())))
    return P, cell, xi
