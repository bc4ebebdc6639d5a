"""Failure detection through status codes (no GPU fault is ever provoked):
bad meshes, non-convergence, degenerate inputs, bad arguments, memory budget."""
import ctypes as C

import numpy as np
import pytest

from synthetic import config_levels
from synthetic.meshes import Level
from tests.oracle_meshes import box_level

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import _abi, nnmg
    return nnmg, _abi


def test_inverted_cell_is_bad_mesh(nn):
    nnmg, _abi = nn
    lv = box_level((3, 3))
    cells = lv.cells.copy()
    cells[4] = cells[4][[1, 0, 3, 2]]              # mirror one cell: negative Jacobian
    bad = Level(2, lv.vertices, cells, lv.dirichlet, lv.n)
    with pytest.raises(nnmg.NNMGError) as e:
        nnmg.Hierarchy([bad], 2)
    assert e.value.status == _abi.BAD_MESH and "Jacobian" in str(e.value)


def test_out_of_range_vertex_index_is_invalid(nn):
    nnmg, _abi = nn
    lv = box_level((2, 2))
    cells = lv.cells.copy()
    cells[0, 0] = 10 ** 6
    with pytest.raises(nnmg.NNMGError) as e:
        nnmg.Hierarchy([Level(2, lv.vertices, cells, lv.dirichlet, lv.n)], 1)
    assert e.value.status == _abi.INVALID_ARG


def test_maxit_reached_reports_not_converged_and_writes_x(nn):
    nnmg, _abi = nn
    H = nnmg.Hierarchy(config_levels("c1_2d_q1"), 1)
    b = H.vector(2, 2)
    H.load_vector(2, np.ones(1), b, col=0)
    H.load_vector(2, np.ones(1) * 2.0, b, col=1)
    x = H.vector(2, 2)
    st, its, rel = H.pcg(b, x, maxit=2, allow_fail=True)
    assert st == _abi.NOT_CONVERGED and np.all(its == 2) and np.all(rel > 1e-8)
    assert torch.count_nonzero(x) > 0
    # a later solve with enough iterations recovers
    st, its, rel = H.pcg(b, x)
    assert st == 0 and np.all(rel <= 1e-8)
    H.close()


def test_zero_rhs_takes_no_iterations(nn):
    nnmg, _abi = nn
    H = nnmg.Hierarchy(config_levels("c1_2d_q1"), 2)
    b = H.vector(2, 3)
    H.load_vector(2, np.ones(1), b, col=1)         # columns 0 and 2 stay zero
    x = H.vector(2, 3) + 5.0
    st, its, rel = H.pcg(b, x)
    assert st == 0 and its[0] == 0 and its[2] == 0 and its[1] > 0
    assert torch.all(x[:, 0] == 0) and torch.all(x[:, 2] == 0)
    H.close()


def test_bad_arguments(nn):
    nnmg, _abi = nn
    lib = _abi.load()
    H = nnmg.Hierarchy(config_levels("c1_2d_q1"), 1, max_nrhs=4)
    x = H.vector(2, 4)
    y = H.vector(2, 4)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    X, Y = C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())
    assert lib.nnmg_apply_operator(H.h, 3, _abi.F64, X, Y, 4, s) == _abi.INVALID_ARG   # level
    assert lib.nnmg_apply_operator(H.h, 2, 9, X, Y, 4, s) == _abi.INVALID_ARG          # precision
    assert lib.nnmg_apply_operator(H.h, 2, _abi.F64, X, Y, 5, s) == _abi.INVALID_ARG   # nrhs > max
    assert lib.nnmg_apply_operator(H.h, 2, _abi.F64, X, X, 4, s) == _abi.INVALID_ARG   # aliasing
    assert lib.nnmg_prolongate(H.h, 0, _abi.F64, X, Y, 4, s) == _abi.INVALID_ARG       # no coarser
    assert lib.nnmg_pcg_solve(H.h, 7, X, Y, 4, 1e-8, 10, None, None, s) == _abi.INVALID_ARG
    assert lib.nnmg_batch_step(H.h, 1, s) == _abi.INVALID_ARG                            # no batch
    assert lib.nnmg_restrict_noalloc(H.h, 0, _abi.F64, X, Y, 4, s) == _abi.INVALID_ARG
    with pytest.raises(ValueError):
        H.apply(2, x[:-1], y[:-1])                                                    # wrong size
    H.close()


def test_serving_budget_too_small_is_refused(nn):
    from paper_2412_10910_gb300.serving import FamilySpec, Server
    srv = Server({"f": FamilySpec(config_levels("c1_2d_q1"), 2)}, budget_bytes=1024)
    with pytest.raises(MemoryError):
        srv.engine("f")
    assert not srv.engines


def test_repeated_solves_agree(nn):
    nnmg, _abi = nn
    H = nnmg.Hierarchy(config_levels("c2_3d_q2", n_levels=3), 2)
    b = H.vector(2, 4)
    b.normal_(generator=torch.Generator(device="cuda").manual_seed(1))
    x1, x2 = H.vector(2, 4), H.vector(2, 4)
    _, i1, _ = H.pcg(b, x1)
    _, i2, _ = H.pcg(b, x2)
    assert np.array_equal(i1, i2)
    assert torch.max(torch.abs(x1 - x2)) <= 1e-12 * torch.max(torch.abs(x1))
    H.close()
