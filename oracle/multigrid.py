"""Smoother, V-cycle (Algorithm 1) and PCG of Sec. 4, on assembled free-DoF matrices.

Solver settings (Sec. 4, list of solver settings), with this project's readings
where the paper is silent:
  * CG in double precision, preconditioned by one V-cycle;
  * V-cycle in single precision (mode "fp32") or double precision ("fp64");
  * Chebyshev iteration of degree m around point Jacobi, eigenvalue estimate
    from 12 Lanczos steps; interval [1.2*lam/20, 1.2*lam] (smoothing range 20,
    safety factor 1.2 - readings);
  * coarsest level: direct solve by a dense Cholesky factorization in FP64
    (the configurations replace the paper's AMG by a direct solve);
  * stopping rule ||r_k||_2 <= rtol ||b||_2 with the recursively updated r.
"""
import numpy as np
import scipy.linalg as sla


def lanczos_start(n_full, free_dofs):
    """Start vector v_i = 1 + 0.01*((i mod 17) - 8) on free DoF indices i (full numbering)."""
    i = np.asarray(free_dofs, dtype=np.int64)
    return 1.0 + 0.01 * ((i % 17) - 8).astype(np.float64)


def lanczos_max_eig(A, D, v0, steps=12):
    """Largest Ritz value of D^-1 A after `steps` Lanczos steps in the D inner product.

    D^-1 A is self-adjoint in <u, v>_D = u^T D v; the three-term recurrence
    builds the tridiagonal T whose largest eigenvalue estimates lambda_max.
    """
    v = v0 / np.sqrt(v0 @ (D * v0))
    v_prev = np.zeros_like(v)
    beta = 0.0
    alphas, betas = [], []
    for j in range(steps):
        w = (A @ v) / D - beta * v_prev
        alpha = w @ (D * v)
        w = w - alpha * v
        beta = np.sqrt(w @ (D * w))
        alphas.append(alpha)
        betas.append(beta)
        if beta == 0.0:
            break
        v_prev, v = v, w / beta
    m = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:m - 1], 1) + np.diag(betas[:m - 1], -1)
    return float(np.max(np.linalg.eigvalsh(T)))


def chebyshev_bounds(lam_max, smoothing_range=20.0, safety=1.2):
    b = safety * lam_max
    return b / smoothing_range, b


def chebyshev(A, Dinv, f, x, m, a, b, x_is_zero):
    """m steps of the Chebyshev iteration for D^-1 A on [a, b] (Saad, Alg. 12.1 form).

    From x = 0 the first residual is f itself, so m-1 operator applications are
    made; otherwise m.  Arithmetic runs in the dtype of the arrays.
    """
    dt = f.dtype
    theta = (a + b) / 2.0
    delta = (b - a) / 2.0
    sigma = theta / delta
    rho = 1.0 / sigma
    r = f.copy() if x_is_zero else f - A @ x
    d = (Dinv * r) / dt.type(theta)
    x = d.copy() if x_is_zero else x + d
    for _ in range(1, m):
        r = f - A @ x
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = dt.type(rho_new * rho) * d + dt.type(2.0 * rho_new / delta) * (Dinv * r)
        x = x + d
        rho = rho_new
    return x


class MGLevel:
    def __init__(self, A, P=None):
        self.A = A                  # free x free CSR, FP64
        self.P = P                  # free fine x free coarse CSR (None on level 1)
        self.D = A.diagonal().copy()
        self.Dinv = 1.0 / self.D
        self.lam = None
        self.bounds = None
        self.f32 = None

    def cast32(self):
        if self.f32 is None:
            self.f32 = dict(A=self.A.astype(np.float32),
                            P=None if self.P is None else self.P.astype(np.float32),
                            Dinv=self.Dinv.astype(np.float32))
        return self.f32


class VCycle:
    """Algorithm 1: pre-smooth from 0, residual, restrict by P^T, recurse, prolongate, post-smooth."""

    def __init__(self, levels, cheb_degree, coarse_factor):
        self.levels = levels        # coarse -> fine
        self.m = cheb_degree
        self.chol = coarse_factor   # scipy cho_factor of A_1

    def coarse_solve(self, f):
        return sla.cho_solve(self.chol, f.astype(np.float64)).astype(f.dtype)

    def __call__(self, f, l=None, precision="fp64"):
        if l is None:
            l = len(self.levels) - 1
        if l == 0:
            return self.coarse_solve(f)
        L = self.levels[l]
        if precision == "fp32":
            c = L.cast32()
            A, Dinv, P = c["A"], c["Dinv"], c["P"]
        else:
            A, Dinv, P = L.A, L.Dinv, L.P
        a, b = L.bounds
        x = chebyshev(A, Dinv, f, None, self.m, a, b, x_is_zero=True)
        r = f - A @ x
        rc = P.T @ r
        dc = self(rc, l - 1, precision)
        x = x + P @ dc
        # Algorithm 1 prints the post-smoother with a zero start; it continues from x.
        x = chebyshev(A, Dinv, f, x, self.m, a, b, x_is_zero=False)
        return x


def pcg(A, b, precond, rtol=1e-8, maxit=200):
    """Preconditioned CG (Hestenes-Stiefel) from x0 = 0 in FP64.

    Returns (x, iterations, relative residual ||r_k||/||b|| of the recursive r,
    true relative residual ||b - A x||/||b||).
    """
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0, 0.0
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rho = r @ z
    it = 0
    rel = 1.0
    while it < maxit:
        q = A @ p
        alpha = rho / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = np.linalg.norm(r) / nb
        if rel <= rtol:
            break
        z = precond(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    true_rel = np.linalg.norm(b - A @ x) / nb
    return x, it, rel, true_rel
