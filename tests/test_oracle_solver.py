"""Pins of the oracle's smoother, eigenvalue estimate, V-cycle and PCG (Sec. 2 Algorithm 1, Sec. 4)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import multigrid
from oracle.hierarchy import OracleHierarchy
from synthetic.meshes import config_levels
from tests.oracle_meshes import box_level


def _cheb_poly(m, lam, a, b):
    """Error polynomial of m Chebyshev steps: T_m((theta-lam)/delta) / T_m(theta/delta)."""
    theta, delta = (a + b) / 2, (b - a) / 2
    t = (theta - lam) / delta
    Tm = np.where(np.abs(t) <= 1, np.cos(m * np.arccos(np.clip(t, -1, 1))),
                  np.cosh(m * np.arccosh(np.maximum(np.abs(t), 1))) * np.sign(t) ** m)
    return Tm / np.cosh(m * np.arccosh(theta / delta))


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_chebyshev_error_reduction_is_closed_form(m):
    lam = np.linspace(0.05, 2.0, 40)
    A = sp.diags(lam).tocsr()
    a, b = 0.1, 1.8
    f = np.linspace(1.0, 2.0, 40)
    xs = A.diagonal() ** -1 * f
    x = multigrid.chebyshev(A, np.ones(40), f, None, m, a, b, x_is_zero=True)
    np.testing.assert_allclose((xs - x) / xs, _cheb_poly(m, lam, a, b), atol=1e-13)
    x0 = np.cos(np.arange(40.0))                        # continuing from a nonzero start
    x = multigrid.chebyshev(A, np.ones(40), f, x0, m, a, b, x_is_zero=False)
    np.testing.assert_allclose((xs - x) / (xs - x0), _cheb_poly(m, lam, a, b), atol=1e-12)


@pytest.mark.parametrize("m", [1, 3, 5])
def test_chebyshev_with_jacobi_scaling_is_closed_form(m):
    """Non-identity diagonal: A = D^(1/2) Q diag(lam) Q^T D^(1/2) with a random
    orthogonal Q, so D^-1 A has eigenvalues lam and eigenvectors D^(-1/2) Q.
    The error of m Chebyshev steps for D^-1 A, written in that eigenbasis
    (coefficients Q^T D^(1/2) e), shrinks by T_m((theta-lam)/delta)/T_m(theta/delta)
    per component (Sec. 4: Chebyshev around point Jacobi).  Passing D where D^-1
    belongs, or dropping the scaling, changes the spectrum the polynomial acts on
    (the diagonal spans two decades here) and fails this."""
    rng = np.random.default_rng(m)
    n = 30
    lam = np.linspace(0.05, 2.0, n)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    dg = 10.0 ** rng.uniform(-1, 1, n)
    sq = np.sqrt(dg)
    A = sp.csr_matrix(sq[:, None] * (Q * lam) @ Q.T * sq[None, :])
    a, b = 0.1, 1.8
    xs = rng.standard_normal(n)
    f = A @ xs
    coeff = lambda e: Q.T @ (sq * e)
    x = multigrid.chebyshev(A, 1.0 / dg, f, None, m, a, b, x_is_zero=True)
    np.testing.assert_allclose(coeff(xs - x) / coeff(xs), _cheb_poly(m, lam, a, b), atol=1e-10)
    x0 = rng.standard_normal(n)
    x = multigrid.chebyshev(A, 1.0 / dg, f, x0, m, a, b, x_is_zero=False)
    np.testing.assert_allclose(coeff(xs - x) / coeff(xs - x0), _cheb_poly(m, lam, a, b), atol=1e-10)


def test_lanczos_exact_when_steps_exceed_dimension():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((9, 9))
    A = B @ B.T + 9 * np.eye(9)
    D = np.abs(np.diag(A)) + rng.random(9)
    lam = sla.eigh(A, np.diag(D), eigvals_only=True).max()
    est = multigrid.lanczos_max_eig(sp.csr_matrix(A), D, rng.random(9) + 0.5, steps=12)
    assert abs(est - lam) < 1e-10 * lam


def test_lanczos_twelve_steps_bounds_lambda_max_from_below():
    H = OracleHierarchy(config_levels("c1_2d_q1"), 1, build_solver=False)
    A = H.A[-1]
    D = A.diagonal()
    v0 = multigrid.lanczos_start(H.levels[-1].n, H.levels[-1].free_dofs)
    est = multigrid.lanczos_max_eig(A, D, v0, 12)
    lam = sla.eigh(A.toarray(), np.diag(D), eigvals_only=True).max()
    assert est <= lam * (1 + 1e-12) and est > 0.95 * lam


def test_coarse_cholesky_solve():
    H = OracleHierarchy(config_levels("c2_3d_q2", n_levels=2), 2)
    A0 = H.A[0].toarray()
    rng = np.random.default_rng(2)
    b = rng.standard_normal(A0.shape[0])
    x = H.vcycle_op.coarse_solve(b)
    assert np.linalg.norm(A0 @ x - b) <= 1e-13 * np.linalg.norm(A0) * np.linalg.norm(x)
    np.testing.assert_allclose(x, np.linalg.solve(A0, b), rtol=1e-10)


@pytest.fixture(scope="module")
def c1():
    return OracleHierarchy(config_levels("c1_2d_q1"), 1, cheb_degree=3)


def test_vcycle_is_symmetric_positive_definite(c1):
    n = len(c1.levels[-1].free_dofs)
    B = np.stack([c1.vcycle_op(e) for e in np.eye(n)], axis=1)
    np.testing.assert_allclose(B, B.T, atol=1e-12 * abs(B).max())
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_vcycle_on_two_identical_levels_reduces_to_smoothing_plus_exact_coarse():
    """Identical coarse and fine meshes: P = I, so the coarse correction solves the
    residual equation exactly and the V-cycle is exact after pre-smoothing; the
    post-smoother then starts at the solution and stays there."""
    lv = box_level((4, 4), alpha=0.2, seed=1)
    H = OracleHierarchy([lv, lv], 2, cheb_degree=3)
    n = len(H.levels[-1].free_dofs)
    f = np.random.default_rng(3).standard_normal(n)
    np.testing.assert_allclose(H.vcycle_op(f), spla.spsolve(H.A[-1].tocsc(), f), rtol=1e-10)


def test_pcg_fixed_point_is_the_direct_solution(c1):
    f = lambda x: (2 * np.pi ** 2 * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]))[:, None]
    b = c1.load_vector(2, f)
    x, its, rel, true = c1.pcg(b, "fp64", rtol=1e-13)
    top = c1.levels[-1]
    xd = spla.spsolve(c1.A[-1].tocsc(), top.to_free(b))
    np.testing.assert_allclose(top.to_free(x), xd, rtol=1e-10, atol=1e-12)
    assert rel[0] <= 1e-13 and true[0] <= 1e-12


def test_mixed_precision_reaches_fp64_accuracy_and_counts_are_close():
    H = OracleHierarchy(config_levels("c2_3d_q2", n_levels=3), 2, cheb_degree=3)
    b = H.load_vector(2, lambda x: np.ones((len(x), 1)))
    x64, it64, r64, _ = H.pcg(b, "fp64", rtol=1e-8)
    x32, it32, r32, t32 = H.pcg(b, "fp32", rtol=1e-8)
    assert r32[0] <= 1e-8 and t32[0] <= 2e-8
    assert abs(it32[0] - it64[0]) <= 1
    assert np.linalg.norm(x32 - x64) <= 1e-7 * np.linalg.norm(x64)
    # roughly constant iteration counts across level counts (Sec. 4)
    H2 = OracleHierarchy(config_levels("c2_3d_q2", n_levels=2), 2, cheb_degree=3)
    b2 = H2.load_vector(1, lambda x: np.ones((len(x), 1)))
    _, it2, _, _ = H2.pcg(b2, "fp32", rtol=1e-8)
    assert abs(it2[0] - it32[0]) <= 3
