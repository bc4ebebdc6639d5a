"""CUDA path vs the FP64 oracle, element by element, on seeded meshes of the
configurations' families (several cell tiles and a ragged last tile each).

Tolerances: FP64 applies (operator, transfers, load vectors) 1e-12 relative
max-norm; FP32 applies 2e-5 relative max-norm (unit roundoff 6e-8 times the
depth of the sum-factorized contraction chains, about 10^2); CG iteration
counts within +-1; the FP32-V-cycle/FP64-CG solution within 1e-7 relative L2
of the FP64 oracle solution after a 1e-8 relative residual.  Integer outputs
(DoF numbering, Dirichlet flags, located coarse cells) are bit-exact.
"""
import numpy as np
import pytest

from tests.gpu_cases import CASES, gpu_case, oracle_case, rng_vec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _relmax(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    name = request.param
    levels, O = oracle_case(name)
    H = gpu_case(name, levels)
    yield name, levels, O, H
    H.close()


def test_numbering_dirichlet_support_points(case):
    name, levels, O, H = case
    for l, lv in enumerate(O.levels):
        np.testing.assert_array_equal(H.cell_nodes(l), lv.node_of)
        np.testing.assert_array_equal(H.constrained(l), lv.constrained)
        np.testing.assert_allclose(H.support_points(l), lv.points, rtol=0, atol=1e-13)


def test_point_location(case):
    name, levels, O, H = case
    for l in range(1, len(O.levels)):
        cell, xi = H.transfer_points(l)
        ocell, oxi = O.loc[l]
        np.testing.assert_array_equal(cell, ocell)
        np.testing.assert_allclose(xi, oxi, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-5), ("dw", 1e-12)])
def test_operator(case, dtype, tol):
    """dw: FP64 vectors, double-word arithmetic (about 2^-48 per operation), held
    to the FP64 tolerance."""
    name, levels, O, H = case
    nrhs = CASES[name][5]
    tdt = torch.float32 if dtype == "f32" else torch.float64
    for l in range(len(O.levels)):
        x = rng_vec(O.levels[l].n, nrhs, 10 + l)
        xo = x.copy()
        xo[np.repeat(O.levels[l].constrained, O.ncomp)] = 0.0
        yo = O.apply(l, xo)
        xt = torch.tensor(x, dtype=tdt, device="cuda")
        y = torch.full_like(xt, 7.0)
        H.apply(l, xt, y, double_word=(dtype == "dw"))
        assert _relmax(y.double().cpu().numpy(), yo) <= tol, (l, _relmax(y.double().cpu().numpy(), yo))


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_prolongation_and_restriction(case, dtype, tol):
    name, levels, O, H = case
    nrhs = CASES[name][5]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    for l in range(1, len(O.levels)):
        xc = rng_vec(O.levels[l - 1].n, nrhs, 20 + l)
        xco = xc.copy()
        xco[np.repeat(O.levels[l - 1].constrained, O.ncomp)] = 0.0
        xf = H.vector(l, nrhs, tdt) + 3.0
        H.prolongate(l, torch.tensor(xc, dtype=tdt, device="cuda"), xf)
        assert _relmax(xf.double().cpu().numpy(), O.prolongate(l, xco)) <= tol
        rf = rng_vec(O.levels[l].n, nrhs, 30 + l)
        rfo = rf.copy()
        rfo[np.repeat(O.levels[l].constrained, O.ncomp)] = 0.0
        rft = torch.tensor(rf, dtype=tdt, device="cuda")
        rc = H.vector(l - 1, nrhs, tdt)
        H.restrict(l, rft, rc)
        ro = O.restrict(l, rfo)
        assert _relmax(rc.double().cpu().numpy(), ro) <= tol
        rc2 = H.vector(l - 1, nrhs, tdt)
        H.restrict(l, rft, rc2)
        assert torch.equal(rc, rc2)            # deterministic, bitwise


def test_eigen_estimates_and_load_vector(case):
    name, levels, O, H = case
    lam = H.eigen_estimates()
    for l in range(1, len(O.levels)):
        assert abs(lam[l] - O.mg[l].lam) <= 1e-9 * O.mg[l].lam
    top = len(O.levels) - 1
    nc = O.ncomp
    fconst = np.arange(1.0, nc + 1.0)
    b = H.vector(top, 2)
    b[:, 1] = 5.0
    H.load_vector(top, fconst, b, col=0)
    bo = O.load_vector(top, lambda x: np.tile(fconst, (len(x), 1)))
    assert _relmax(b[:, 0].cpu().numpy(), bo) <= 1e-12
    assert torch.all(b[:, 1] == 5.0)


def test_vcycle(case):
    name, levels, O, H = case
    nrhs = CASES[name][5]
    top = len(O.levels) - 1
    r = rng_vec(O.levels[top].n, nrhs, 40)
    ro = r.copy()
    ro[np.repeat(O.levels[top].constrained, O.ncomp)] = 0.0
    zo = O.vcycle(ro, "fp64")
    z = H.vector(top, nrhs)
    H.vcycle(torch.tensor(r, device="cuda"), z)
    assert _relmax(z.cpu().numpy(), zo) <= 1e-9
    # FP32 V-cycle against the oracle's V-cycle run in float arithmetic (the same
    # Algorithm 1 on float CSR matrices).  The two round differently; on these
    # cases the oracle's FP32 and FP64 V-cycles differ by 1e-7 .. 2e-6 relative
    # max-norm, so both distances are held to the FP32 apply tolerance.
    r32 = torch.tensor(r, dtype=torch.float32, device="cuda")
    zo32 = O.vcycle(r32.double().cpu().numpy(), "fp32")
    z32 = H.vector(top, nrhs, torch.float32)
    H.vcycle(r32, z32)
    z32 = z32.double().cpu().numpy()
    assert _relmax(z32, zo32) <= 2e-5, _relmax(z32, zo32)
    assert _relmax(z32, zo) <= 2e-5, _relmax(z32, zo)
    z2 = H.vector(top, nrhs)                   # second call replays the captured graph
    H.vcycle(torch.tensor(r, device="cuda"), z2)
    assert _relmax(z2.cpu().numpy(), zo) <= 1e-9


@pytest.mark.parametrize("mode", ["fp32", "fp64", "dw"])
def test_pcg(case, mode):
    from paper_2412_10910_gb300 import _abi
    name, levels, O, H = case
    nrhs = CASES[name][5]
    top = len(O.levels) - 1
    n = O.levels[top].n
    b = rng_vec(n, nrhs, 50)
    b[np.repeat(O.levels[top].constrained, O.ncomp)] = 0.0
    xo64, its64, _, _ = O.pcg(b, "fp64", rtol=1e-8)
    _, itso, _, _ = O.pcg(b, "fp32" if mode == "dw" else mode, rtol=1e-8)
    bt = torch.tensor(b, device="cuda")
    x = H.vector(top, nrhs)
    m = {"fp32": _abi.FP32_MG_FP64_CG, "fp64": _abi.FP64_MG, "dw": _abi.FP32_MG_DW_CG}[mode]
    for rep in range(2):                       # eager first call, graph replay second
        st, its, rel = H.pcg(bt, x, mode=m, rtol=1e-8, maxit=100)
        assert st == 0 and np.all(rel <= 1e-8)
        assert np.all(np.abs(its - np.array(itso)) <= 1), (its, itso)
        xs = x.cpu().numpy()
        err = np.linalg.norm(xs - xo64, axis=0) / np.linalg.norm(xo64, axis=0)
        assert np.all(err <= 1e-7), err
