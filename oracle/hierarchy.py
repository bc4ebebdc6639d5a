"""A whole oracle hierarchy: numbering, assembled operators, transfers, V-cycle, PCG.

Vectors at this interface are full length (n_nodes * ncomp, node-major) with
zeros at Dirichlet DoFs, the layout of the GPU library's interface; the
matrices themselves act on free DoFs only.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import dofs, assembly, transfer, multigrid


class OracleLevel:
    def __init__(self, lv, k, ncomp, lame):
        self.dim = lv.dim
        self.vertices = lv.vertices
        self.cells = lv.cells
        self.k = k
        self.ncomp = ncomp
        self.node_of, self.n_nodes, oc, ol = dofs.number_dofs(lv.cells, k, lv.dim)
        self.constrained = dofs.dirichlet_nodes(lv.cells, lv.dirichlet, self.node_of, k, lv.dim)
        self.free_nodes = np.nonzero(~self.constrained)[0]
        self.points = dofs.support_points(lv.vertices, lv.cells, oc, ol, k, lv.dim)
        free_dof_mask = np.repeat(~self.constrained, ncomp)
        self.free_dofs = np.nonzero(free_dof_mask)[0]
        self.n = self.n_nodes * ncomp
        self.lame = lame
        self._A_full = None

    def assemble(self):
        elem = assembly.element_matrices(self.vertices, self.cells, self.k, self.dim,
                                         self.ncomp, self.lame)
        A = assembly.assemble(elem, self.node_of, self.n_nodes, self.ncomp)
        self._A_full = A
        fd = self.free_dofs
        return A[fd][:, fd].tocsr()

    def to_free(self, v):
        return v[self.free_dofs]

    def to_full(self, vf):
        out = np.zeros((self.n,) + vf.shape[1:], dtype=vf.dtype)
        out[self.free_dofs] = vf
        return out


class OracleHierarchy:
    def __init__(self, levels, degree, ncomp=1, lame=(1.0, 1.0), cheb_degree=3,
                 lanczos_steps=12, smoothing_range=20.0, safety=1.2, build_solver=True,
                 level_degrees=None):
        """level_degrees: optional per-level degrees (0 = degree), coarse -> fine; repeating
        the coarsest mesh with degrees 1..k gives polynomial coarsening on that mesh
        (Sec. 2, "Coarse grid solvers")."""
        self.degree = degree
        self.ncomp = ncomp
        degs = [d or degree for d in (level_degrees or [0] * len(levels))]
        self.levels = [OracleLevel(lv, k, ncomp, lame) for lv, k in zip(levels, degs)]
        self.A = [lv.assemble() for lv in self.levels]
        self.P = [None]
        self.loc = [None]
        for l in range(1, len(self.levels)):
            f, c = self.levels[l], self.levels[l - 1]
            cd = dict(vertices=c.vertices, cells=c.cells, node_of=c.node_of, free=~c.constrained)
            Pn, cell, xi = transfer.transfer_matrix(f.points, f.free_nodes, cd, c.k, f.dim)
            Pd = sp.kron(Pn, sp.identity(ncomp), format="csr") if ncomp > 1 else Pn
            self.P.append(Pd.tocsr())
            self.loc.append((cell, xi))
        self.cheb_degree = cheb_degree
        if build_solver:
            self.mg = [multigrid.MGLevel(self.A[l], self.P[l]) for l in range(len(self.levels))]
            for l in range(1, len(self.levels)):
                L = self.mg[l]
                v0 = multigrid.lanczos_start(self.levels[l].n, self.levels[l].free_dofs)
                L.lam = multigrid.lanczos_max_eig(L.A, L.D, v0, lanczos_steps)
                L.bounds = multigrid.chebyshev_bounds(L.lam, smoothing_range, safety)
            self.chol = sla.cho_factor(self.A[0].toarray(), lower=True)
            self.vcycle_op = multigrid.VCycle(self.mg, cheb_degree, self.chol)

    # ---- full-length vector helpers (columns = right-hand sides) ----
    def apply(self, l, x):
        lv = self.levels[l]
        return lv.to_full(self.A[l] @ lv.to_free(x))

    def prolongate(self, l_fine, xc):
        f, c = self.levels[l_fine], self.levels[l_fine - 1]
        return f.to_full(self.P[l_fine] @ c.to_free(xc))

    def restrict(self, l_fine, rf):
        f, c = self.levels[l_fine], self.levels[l_fine - 1]
        return c.to_full(self.P[l_fine].T @ f.to_free(rf))

    def vcycle(self, r, precision="fp64"):
        top = self.levels[-1]
        rf = top.to_free(r)
        cols = rf.reshape(rf.shape[0], -1)
        dt = np.float32 if precision == "fp32" else np.float64
        out = np.stack([self.vcycle_op(cols[:, j].astype(dt), precision=precision)
                        for j in range(cols.shape[1])], axis=1)
        return top.to_full(out.astype(np.float64).reshape(rf.shape))

    def pcg(self, b, mode="fp32", rtol=1e-8, maxit=200):
        """Solve every column of b; returns (x, iters[list], relres[list], true_relres[list])."""
        top = self.levels[-1]
        A = self.A[-1]
        bf = top.to_free(b).reshape(top.free_dofs.size, -1)
        prec = "fp32" if mode == "fp32" else "fp64"
        dt = np.float32 if prec == "fp32" else np.float64

        def M(r):
            return self.vcycle_op(r.astype(dt), precision=prec).astype(np.float64)

        xs, its, rels, trues = [], [], [], []
        for j in range(bf.shape[1]):
            x, it, rel, tr = multigrid.pcg(A, bf[:, j].copy(), M, rtol, maxit)
            xs.append(x); its.append(it); rels.append(rel); trues.append(tr)
        X = np.stack(xs, axis=1)
        return top.to_full(X).reshape(b.shape), its, rels, trues

    def load_vector(self, l, f):
        lv = self.levels[l]
        b = assembly.load_vector(lv.vertices, lv.cells, lv.node_of, lv.n_nodes, lv.k,
                                 lv.dim, f, lv.ncomp)
        b[np.repeat(lv.constrained, lv.ncomp)] = 0.0
        return b
