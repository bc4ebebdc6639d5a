"""Element matrices, assembled CSR operators and load vectors in FP64.

Poisson (Sec. 2, Eq. problem with a(u,v) = (grad u, grad v)):
    A_K[i,j] = sum_q w_q |det J| (J^-T grad^ phi_i) . (J^-T grad^ phi_j)
Linear elasticity (Sec. 4.4, Eq. linear_elasticity; sigma = lambda tr(eps) I + 2 mu eps):
    a(u,v) = sum_q w_q |det J| [lambda div u div v + 2 mu eps(u):eps(v)]
    which for u = phi_j e_e, v = phi_i e_c reads
    lambda d_c phi_i d_e phi_j + mu (delta_ce grad phi_i . grad phi_j + d_e phi_i d_c phi_j).
Quadrature: Gauss-Legendre with (k+1)^d points (Sec. 4).
"""
import numpy as np
import scipy.sparse as sp

from .fe import tensor_quadrature, tensor_basis, q1_shape


def geometry(vertices, cells, dim, qpts):
    """Jacobians J[c,q,a,b] = dx_a/dxi_b, determinants, inverses and x_q."""
    N, dN = q1_shape(dim, qpts)                       # [nq, nv], [nq, nv, dim]
    X = vertices[cells]                               # [nc, nv, dim]
    J = np.einsum("cva,qvb->cqab", X, dN)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    xq = np.einsum("qv,cva->cqa", N, X)
    return J, det, Jinv, xq


def element_matrices(vertices, cells, k, dim, ncomp=1, lame=(1.0, 1.0), chunk=4096):
    """Local matrices [nc, nloc*ncomp, nloc*ncomp] (node-major, component inner)."""
    qpts, qw = tensor_quadrature(k + 1, dim)
    _, gref = tensor_basis(k, dim, qpts)              # [nq, nloc, dim]
    nc = cells.shape[0]
    nloc = gref.shape[1]
    out = np.empty((nc, nloc * ncomp, nloc * ncomp))
    lam, mu = lame
    for c0 in range(0, nc, chunk):
        cs = slice(c0, min(nc, c0 + chunk))
        J, det, Jinv, _ = geometry(vertices, cells[cs], dim, qpts)
        if np.any(det <= 0):
            raise ValueError("non-positive Jacobian determinant")
        dw = det * qw[None, :]                        # [c, q]
        # physical gradients g[c,q,i,b] = sum_a gref[q,i,a] Jinv[c,q,a,b]
        g = np.einsum("qia,cqab->cqib", gref, Jinv)
        if ncomp == 1:
            out[cs] = np.einsum("cq,cqia,cqja->cij", dw, g, g)
        else:
            ncq = g.shape[0]
            blk = np.zeros((ncq, nloc, ncomp, nloc, ncomp))
            gg = np.einsum("cq,cqia,cqja->cij", dw, g, g)
            for c in range(ncomp):
                for e in range(ncomp):
                    t = lam * np.einsum("cq,cqi,cqj->cij", dw, g[..., c], g[..., e])
                    t += mu * np.einsum("cq,cqi,cqj->cij", dw, g[..., e], g[..., c])
                    if c == e:
                        t += mu * gg
                    blk[:, :, c, :, e] = t
            out[cs] = blk.reshape(ncq, nloc * ncomp, nloc * ncomp)
    return out


def assemble(elem, node_of, n_nodes, ncomp=1):
    """Global CSR matrix over all DoFs (node*ncomp + comp) from local matrices."""
    nc, m, _ = elem.shape
    if ncomp == 1:
        gd = node_of
    else:
        gd = (node_of[:, :, None] * ncomp + np.arange(ncomp)[None, None, :]).reshape(nc, -1)
    rows = np.repeat(gd, m, axis=1).ravel()
    cols = np.tile(gd, (1, m)).ravel()
    n = n_nodes * ncomp
    A = sp.coo_matrix((elem.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def load_vector(vertices, cells, node_of, n_nodes, k, dim, f, ncomp=1):
    """b_(i,c) = sum_K sum_q w_q |det J| f_c(x_q) phi_i(xi_q); f maps [P,dim] -> [P,ncomp]."""
    qpts, qw = tensor_quadrature(k + 1, dim)
    val, _ = tensor_basis(k, dim, qpts)               # [nq, nloc]
    J, det, _, xq = geometry(vertices, cells, dim, qpts)
    nc, nq, _ = xq.shape
    fq = np.asarray(f(xq.reshape(-1, dim)), dtype=np.float64).reshape(nc, nq, ncomp)
    contrib = np.einsum("cq,qi,cqe->cie", det * qw[None, :], val, fq)    # [nc, nloc, ncomp]
    b = np.zeros(n_nodes * ncomp)
    idx = (node_of[:, :, None] * ncomp + np.arange(ncomp)[None, None, :])
    np.add.at(b, idx.ravel(), contrib.ravel())
    return b


def quadrature_points(vertices, cells, k, dim):
    """Physical quadrature points [nc, (k+1)^d, dim]."""
    qpts, _ = tensor_quadrature(k + 1, dim)
    _, _, _, xq = geometry(vertices, cells, dim, qpts)
    return xq
