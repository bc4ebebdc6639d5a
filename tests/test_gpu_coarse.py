"""The coarsest level's direct solve (Algorithm 1: delta_1 = A_1^-1 r_1), whose
dense operator and inverse are built on the device at setup.

A one-level hierarchy's V-cycle is exactly that solve, so it is compared with
numpy's dense solve of the oracle's assembled free-DoF matrix (FP64, 1e-10
relative max-norm).  The sizes span one partial pivot block (16 free rows)
to 3375 free rows (52 full blocks of 64 and a ragged one), Poisson and
elasticity.
"""
import numpy as np
import pytest

from synthetic import config_levels

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# name -> (levels, degree, ncomp, lame, nrhs)
COARSE = {
    "c1_coarsest_q1": (lambda: config_levels("c1_2d_q1", n_levels=1), 1, 1, (1.0, 1.0), 3),
    "c2_coarsest_q2": (lambda: config_levels("c2_3d_q2", n_levels=1), 2, 1, (1.0, 1.0), 8),
    "c3_coarsest_q4": (lambda: config_levels("c3_3d_q4_deformed", n_levels=1), 4, 1, (1.0, 1.0), 4),
    "c4_coarsest_q2": (lambda: config_levels("c4_3d_q2_elasticity", n_levels=1), 2, 3, (10.0, 1.0), 2),
}


@pytest.mark.parametrize("name", list(COARSE))
def test_direct_coarse_solve_matches_dense_solve(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.hierarchy import OracleHierarchy
    from paper_2412_10910_gb300 import nnmg
    lv, k, nc, lame, nrhs = COARSE[name]
    levels = lv()
    O = OracleHierarchy(levels, k, nc, lame, build_solver=False)
    top = O.levels[0]
    A = O.A[0].toarray()
    rng = np.random.default_rng(3)
    r = rng.standard_normal((top.n, nrhs))
    r[np.repeat(top.constrained, nc)] = 0.0
    ref = top.to_full(np.linalg.solve(A, top.to_free(r)))
    H = nnmg.Hierarchy(levels, k, nc, lame, max_nrhs=16)
    try:
        z = H.vector(0, nrhs)
        H.vcycle(torch.tensor(r, device="cuda"), z)
        z = z.cpu().numpy()
        err = np.max(np.abs(z - ref)) / np.max(np.abs(ref))
        assert err <= 1e-10, err
    finally:
        H.close()
