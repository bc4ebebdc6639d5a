"""The per-level V-cycle profile (the component breakdown of the paper's
Sec. 5, Fig. breakdown_serial) runs the same kernels as nnmg_vcycle.

Its z equals nnmg_vcycle's up to the rounding of the operator's
floating-point atomics, every component it reports was timed, the component
columns and the kernel-class columns book the same launches, and the launch
counts follow Algorithm 1 with a degree-m Chebyshev smoother: m - 1 operator
passes before the residual's, m after the prolongation.  The residual's
subtraction runs inside the restriction's first kernel, so the residual
column books the operator pass alone; where the persistent smoother serves a
level, each smoothing sweep (the pre-smoothing one with the residual's
operator pass) is one launch.
"""
import numpy as np
import pytest

from tests.gpu_cases import CASES, gpu_case, oracle_case, rng_vec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name", ["c1_q1", "c2_q2_3lev", "c4_elast"])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_profile_matches_vcycle_and_books_every_launch(name, dtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import _abi
    levels, O = oracle_case(name)
    _, k, nc, lame, m, nrhs = CASES[name][:6]
    H = gpu_case(name, levels)
    try:
        top = H.n_levels - 1
        dt = getattr(torch, dtype)
        r = torch.tensor(rng_vec(H.rows(top), nrhs, 7), dtype=dt, device="cuda")
        r[torch.tensor(np.repeat(H.constrained(top), nc), device="cuda")] = 0
        z_ref = torch.empty_like(r)
        H.vcycle(r, z_ref)
        z = torch.full_like(r, float("nan"))
        ms, cnt = H.vcycle_profile(r, z)
        torch.cuda.synchronize()
        tol = 1e-5 if dtype == "float32" else 1e-12
        err = (z - z_ref).norm() / z_ref.norm()
        assert float(err) <= tol, float(err)

        col = {c: i for i, c in enumerate(_abi.PROF_COLUMNS)}
        assert ms.shape == (H.n_levels, len(_abi.PROF_COLUMNS))
        assert cnt[0, col["coarse_solver"]] == 1 and ms[0, col["coarse_solver"]] > 0
        assert cnt[0].sum() == 1
        for lv in range(1, H.n_levels):
            c = cnt[lv]
            assert c[col["restrictor"]] == 1 and c[col["prolongator"]] == 1
            assert c[col["coarse_solver"]] == 0
            if c[col["pre_smoother"]] == 1:
                # persistent smoother: one launch per sweep, the pre-smoothing
                # one ending with the residual's operator pass
                assert c[col["residual"]] == 0 and c[col["post_smoother"]] == 1
                assert c[col["operator"]] == 2 and c[col["vector"]] == 0
            else:
                assert c[col["pre_smoother"]] == 1 + 2 * (m - 1)
                assert c[col["residual"]] == 1
                assert c[col["post_smoother"]] == 2 * m
                assert c[col["operator"]] == 2 * m
                assert c[col["vector"]] == 2 * m
            assert (ms[lv, :6][c[:6] > 0] > 0).all()
            # the two views of a level book the same smoother and residual time
            smooth = ms[lv, col["pre_smoother"]] + ms[lv, col["residual"]] + ms[lv, col["post_smoother"]]
            assert abs(smooth - ms[lv, col["operator"]] - ms[lv, col["vector"]]) <= 1e-9 * max(1.0, smooth)
    finally:
        H.close()


def test_profile_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes as C

    from paper_2412_10910_gb300 import _abi
    levels, O = oracle_case("c1_q1")
    H = gpu_case("c1_q1", levels)
    try:
        top = H.n_levels - 1
        r = torch.zeros(H.rows(top), 1, dtype=torch.float32, device="cuda")
        z = torch.empty_like(r)
        lib = _abi.load()
        s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        ms = np.zeros((H.n_levels, len(_abi.PROF_COLUMNS)))
        assert lib.nnmg_vcycle_profile(H.h, _abi.F32, C.c_void_p(r.data_ptr()),
                                       C.c_void_p(z.data_ptr()), 1, s, None, None) == _abi.INVALID_ARG
        assert lib.nnmg_vcycle_profile(H.h, _abi.F32, C.c_void_p(r.data_ptr()),
                                       C.c_void_p(z.data_ptr()), 0, s, ms.ctypes.data,
                                       None) == _abi.INVALID_ARG
        # launches may be NULL
        assert lib.nnmg_vcycle_profile(H.h, _abi.F32, C.c_void_p(r.data_ptr()),
                                       C.c_void_p(z.data_ptr()), 1, s, ms.ctypes.data, None) == 0
        assert ms[0, 3] > 0
    finally:
        H.close()
