"""nnmg_restrict_noalloc against nnmg_restrict, through the C interface.

The no-allocation variant serves callers that may not allocate device memory
while they run (allocator-free real-time loops, externally budgeted memory,
host callbacks): it takes its scratch from a fixed array inside the library.
Both entry points run the same deterministic two-phase gather, so their
results must be bitwise equal.  This file is collected last, and it builds its
own hierarchies, so it passes alone in a fresh process and after the other
tests.
"""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LEVELS = dict(name="c2_3d_q2", n_levels=3)


def _levels():
    from synthetic import config_levels
    return config_levels(LEVELS["name"], n_levels=LEVELS["n_levels"])


@pytest.fixture(scope="module")
def hier():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import nnmg
    H = nnmg.Hierarchy(_levels(), 2, cheb_degree=3, max_nrhs=16)
    yield H
    H.close()


def _ptr(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_restriction_equals_allocating_one_twice(hier, dtype):
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
            assert lib.nnmg_restrict(hier.h, fine_level, prec, _ptr(rf), _ptr(ref), nrhs, stream) == 0
            st = lib.nnmg_restrict_noalloc(hier.h, fine_level, prec, _ptr(rf), _ptr(out), nrhs, stream)
            assert st == 0, nnmg.nnmg_last_error()
            torch.cuda.synchronize()
            assert torch.equal(out, ref)


def test_first_call_on_a_fresh_hierarchy_allocates_nothing():
    """nnmg_restrict_noalloc first, on a hierarchy that has run nothing yet:
    device free memory is unchanged across the call, and the result equals
    nnmg_restrict's (called afterwards, which allocates its own buffers)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import _abi, nnmg
    lib = _abi.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    nrhs, fl = 8, 2
    # load the restriction kernels once on another hierarchy, so the driver's
    # lazy module loading does not count against the call below
    warm = nnmg.Hierarchy(_levels(), 2, cheb_degree=3, max_nrhs=16)
    for dt in (torch.float64, torch.float32):
        wf = torch.zeros(warm.rows(fl), nrhs, dtype=dt, device="cuda")
        wc = warm.vector(fl - 1, nrhs, dt)
        assert lib.nnmg_restrict(warm.h, fl, _abi.F64 if dt == torch.float64 else _abi.F32,
                                 _ptr(wf), _ptr(wc), nrhs, stream) == 0
    torch.cuda.synchronize()
    H = nnmg.Hierarchy(_levels(), 2, cheb_degree=3, max_nrhs=16)
    for dt, prec in ((torch.float64, _abi.F64), (torch.float32, _abi.F32)):
        g = torch.Generator(device="cuda").manual_seed(7)
        rf = torch.randn(H.rows(fl), nrhs, dtype=dt, device="cuda", generator=g)
        out = torch.full((H.rows(fl - 1), nrhs), float("nan"), dtype=dt, device="cuda")
        ref = torch.zeros_like(out)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            st = lib.nnmg_restrict_noalloc(H.h, fl, prec, _ptr(rf), _ptr(out), nrhs, stream)
            assert st == 0, nnmg.nnmg_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert lib.nnmg_restrict(H.h, fl, prec, _ptr(rf), _ptr(ref), nrhs, stream) == 0
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    H.close()
    warm.close()


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
    st = lib.nnmg_restrict_noalloc(H.h, 3, _abi.F64, _ptr(rf), _ptr(rc), 16, None)
    assert st == _abi.INVALID_ARG and b"scratch" in lib.nnmg_last_error()
    H.close()
