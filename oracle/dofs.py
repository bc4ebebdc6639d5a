"""Continuous Q_k DoF numbering, Dirichlet set and support points (Sec. 2).

Numbering rule (the vector layout shared with the GPU library's interface):
each local node of a cell is identified by the multilinear combination of the
cell's corner vertices that places it, using the equispaced proxy m/k for the
Gauss-Lobatto position of node index m (the Gauss-Lobatto set is symmetric, so
the proxy identifies the same node from every cell sharing it).  Nodes receive
ids in order of first appearance, walking cells in index order and each cell's
local nodes lexicographically (x fastest).  A vector-valued field stores the
components of a node contiguously: index = node * n_components + component.

Dirichlet set: every node that lies on a boundary face (a face of exactly one
cell) whose corner vertices are all flagged.
"""
import numpy as np

from .fe import multi_indices, gauss_lobatto_nodes, q1_shape


def corner_weights(k: int, dim: int) -> np.ndarray:
    """Integer weights W[i, v] = prod_d (m_d if bit_d(v) else k - m_d), [nloc, 2^d]."""
    mi = multi_indices(k + 1, dim)
    nv = 2 ** dim
    W = np.ones((len(mi), nv), dtype=np.int64)
    for v in range(nv):
        for d in range(dim):
            bit = (v >> d) & 1
            W[:, v] *= mi[:, d] if bit else (k - mi[:, d])
    return W


def number_dofs(cells: np.ndarray, k: int, dim: int):
    """Return (cell_nodes [nc, nloc], n_nodes, owner_cell [n], owner_local [n])."""
    nc = cells.shape[0]
    W = corner_weights(k, dim)                           # [nloc, nv]
    nloc, nv = W.shape
    big = np.iinfo(np.int64).max
    vid = np.where(W[None, :, :] != 0, cells[:, None, :].astype(np.int64), big)  # [nc, nloc, nv]
    wts = np.broadcast_to(W[None], vid.shape)
    order = np.argsort(vid, axis=2, kind="stable")
    vs = np.take_along_axis(vid, order, axis=2)
    ws = np.take_along_axis(wts, order, axis=2)
    ws = np.where(vs == big, 0, ws)
    keys = np.concatenate([vs, ws], axis=2).reshape(nc * nloc, 2 * nv)
    uniq, first, inverse = np.unique(keys, axis=0, return_index=True, return_inverse=True)
    inverse = inverse.reshape(-1)
    # ids in order of first appearance
    rank = np.empty(len(uniq), dtype=np.int64)
    rank[np.argsort(first, kind="stable")] = np.arange(len(uniq))
    node_of = rank[inverse].reshape(nc, nloc)
    owner = np.empty(len(uniq), dtype=np.int64)
    owner[rank] = first
    return node_of, len(uniq), owner // nloc, owner % nloc


def cell_faces(dim: int):
    """Faces of the reference cell as (direction a, side s, corner list)."""
    faces = []
    for a in range(dim):
        for s in (0, 1):
            corners = [v for v in range(2 ** dim) if ((v >> a) & 1) == s]
            faces.append((a, s, corners))
    return faces


def dirichlet_nodes(cells, dirichlet_vertex, node_of, k, dim) -> np.ndarray:
    """Boolean mask over nodes: on a boundary face whose corners are all flagged."""
    nc = cells.shape[0]
    mi = multi_indices(k + 1, dim)
    faces = cell_faces(dim)
    fkeys = []
    for (a, s, corners) in faces:
        fkeys.append(np.sort(cells[:, corners].astype(np.int64), axis=1))
    allkeys = np.concatenate(fkeys, axis=0)
    _, inv, counts = np.unique(allkeys, axis=0, return_inverse=True, return_counts=True)
    inv = inv.reshape(-1)
    is_boundary = counts[inv] == 1
    n_nodes = node_of.max() + 1
    mask = np.zeros(n_nodes, dtype=bool)
    for f, (a, s, corners) in enumerate(faces):
        sel = slice(f * nc, (f + 1) * nc)
        flagged = np.all(dirichlet_vertex[cells[:, corners]] != 0, axis=1)
        hit = is_boundary[sel] & flagged
        on_face = np.nonzero(mi[:, a] == s * k)[0]
        mask[node_of[hit][:, on_face].ravel()] = True
    return mask


def support_points(vertices, cells, owner_cell, owner_local, k, dim) -> np.ndarray:
    """x_i = F_K(xi_i) evaluated in the first cell that numbered node i, [n, dim]."""
    nodes = gauss_lobatto_nodes(k)
    mi = multi_indices(k + 1, dim)
    xi = nodes[mi[owner_local]]                            # [n, dim]
    N, _ = q1_shape(dim, xi)                               # [n, nv]
    X = vertices[cells[owner_cell]]                        # [n, nv, dim]
    return np.einsum("pv,pvd->pd", N, X)
