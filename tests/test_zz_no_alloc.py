"""nnmg_restrict_noalloc against nnmg_restrict, through the C interface.

The no-allocation variant serves callers that may not allocate device memory
while they run (allocator-free real-time loops, externally budgeted memory,
host callbacks): it takes its scratch from a fixed array inside the library.
Its results must equal those of nnmg_restrict.  This file is collected last,
and it builds its own hierarchy, so it passes alone in a fresh process and
after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hier():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import nnmg
    from synthetic import config_levels
    H = nnmg.Hierarchy(config_levels("c2_3d_q2", n_levels=3), 2, cheb_degree=3, max_nrhs=16)
    yield H
    H.close()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_noalloc_restriction_matches_allocating_one_twice(hier, dtype, tol):
    from paper_2412_10910_gb300 import _abi, nnmg
    lib = _abi.load()
    prec = _abi.F64 if dtype == torch.float64 else _abi.F32
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for fine_level, nrhs, seed in [(2, 8, 1), (2, 3, 2), (1, 16, 3)]:
        for call in range(2):                       # two calls in a row, fresh inputs
            g = torch.Generator(device="cuda").manual_seed(100 * seed + call)
            rf = torch.randn(hier.rows(fine_level), nrhs, dtype=dtype, device="cuda", generator=g)
            ref = hier.vector(fine_level - 1, nrhs, dtype)
            out = torch.full_like(ref, float("nan"))
            assert lib.nnmg_restrict(hier.h, fine_level, prec, C.c_void_p(rf.data_ptr()),
                                     C.c_void_p(ref.data_ptr()), nrhs, stream) == 0
            st = lib.nnmg_restrict_noalloc(hier.h, fine_level, prec, C.c_void_p(rf.data_ptr()),
                                           C.c_void_p(out.data_ptr()), nrhs, stream)
            assert st == 0, nnmg.nnmg_last_error()
            torch.cuda.synchronize()
            a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
            assert np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(b)), 1e-300)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import _abi, nnmg
    from synthetic import config_levels
    lib = _abi.load()
    # 55^3 fine level onto 27^3 coarse cells: 19683 x 27 x 16 x 8 B = 68 MB > 64 MiB
    H = nnmg.Hierarchy(config_levels("c2_3d_q2"), 2, cheb_degree=3, max_nrhs=16)
    rf = torch.zeros(H.rows(3), 16, dtype=torch.float64, device="cuda")
    rc = torch.zeros(H.rows(2), 16, dtype=torch.float64, device="cuda")
    st = lib.nnmg_restrict_noalloc(H.h, 3, _abi.F64, C.c_void_p(rf.data_ptr()),
                                   C.c_void_p(rc.data_ptr()), 16, None)
    assert st == _abi.INVALID_ARG and b"scratch" in lib.nnmg_last_error()
    H.close()
