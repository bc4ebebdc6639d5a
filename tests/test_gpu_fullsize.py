"""Full-size parity: configuration 2 (the benchmark's launch configuration:
3D Q2, 55^3 fine cells, 8 right-hand sides) and configuration 3 (3D Q4 on the
deformed cube, 39^3 fine cells, 4 right-hand sides).

At these sizes the oracle computes sampled outputs one by one: the DoF
numbering of the whole fine mesh, operator rows from the element matrices of
the cells around sampled nodes, located points and prolongated values at
sampled fine nodes.  Properties that hold at any size cover the rest:
<P x, y> = <x, P^T y> for restriction, the true residual of the PCG solution
and the agreement of the two precision modes.  Tolerances as in
test_gpu_parity.py.
"""
import numpy as np
import pytest

from oracle import assembly, dofs, fe, transfer
from synthetic import config_levels
from synthetic.meshes import CONFIGS

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FULL = ["c2_3d_q2", "c3_3d_q4_deformed"]


@pytest.fixture(scope="module", params=FULL)
def full(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import nnmg
    name = request.param
    cfg = CONFIGS[name]
    levels = config_levels(name)
    H = nnmg.Hierarchy(levels, cfg["degree"], 1, cheb_degree=cfg["cheb"], max_nrhs=16)
    top = len(levels) - 1
    f = levels[top]
    node_of, nn, oc, ol = dofs.number_dofs(f.cells, cfg["degree"], 3)
    cons = dofs.dirichlet_nodes(f.cells, f.dirichlet, node_of, cfg["degree"], 3)
    pts = dofs.support_points(f.vertices, f.cells, oc, ol, cfg["degree"], 3)
    yield name, cfg, levels, H, node_of, nn, cons, pts
    H.close()


def test_fine_numbering_bit_exact(full):
    name, cfg, levels, H, node_of, nn, cons, pts = full
    top = len(levels) - 1
    np.testing.assert_array_equal(H.cell_nodes(top), node_of)
    np.testing.assert_array_equal(H.constrained(top), cons)
    np.testing.assert_allclose(H.support_points(top), pts, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_operator_sampled_rows(full, dtype, tol):
    name, cfg, levels, H, node_of, nn, cons, pts = full
    top = len(levels) - 1
    f = levels[top]
    nrhs, k = cfg["nrhs"], cfg["degree"]
    rng = np.random.default_rng(7)
    x = rng.standard_normal((nn, nrhs))
    x[cons] = 0.0
    tdt = torch.float64 if dtype == "f64" else torch.float32
    xt = torch.tensor(x, dtype=tdt, device="cuda")
    y = torch.empty_like(xt)
    H.apply(top, xt, y)
    y = y.double().cpu().numpy()
    xin = xt.double().cpu().numpy()        # the exact input the kernel saw
    sample = rng.choice(np.nonzero(~cons)[0], 300, replace=False)
    cells = np.unique(np.nonzero(np.isin(node_of, sample))[0])
    E = assembly.element_matrices(f.vertices, f.cells[cells], k, 3)
    yo = np.zeros((nn, nrhs))
    for c, Ec in zip(cells, E):
        loc = node_of[c]
        yo[loc] += Ec @ xin[loc]
    ref = yo[sample]
    scale = np.max(np.abs(y))
    assert np.max(np.abs(y[sample] - ref)) <= tol * scale
    assert np.all(y[cons] == 0.0)


def test_point_location_and_prolongation_sampled(full):
    name, cfg, levels, H, node_of, nn, cons, pts = full
    top = len(levels) - 1
    c = levels[top - 1]
    k, nrhs = cfg["degree"], cfg["nrhs"]
    cnode, cnn, _, _ = dofs.number_dofs(c.cells, k, 3)
    ccons = dofs.dirichlet_nodes(c.cells, c.dirichlet, cnode, k, 3)
    cell, xi = H.transfer_points(top)
    free = np.nonzero(~cons)[0]
    rng = np.random.default_rng(11)
    sel = rng.choice(len(free), 300, replace=False)
    ocell, oxi = transfer.locate(pts[free[sel]], c.vertices, c.cells, 3)
    np.testing.assert_array_equal(cell[sel], ocell)
    np.testing.assert_allclose(xi[sel], oxi, rtol=0, atol=1e-12)
    xc = rng.standard_normal((cnn, nrhs))
    xc[ccons] = 0.0
    xf = H.vector(top, nrhs)
    H.prolongate(top, torch.tensor(xc, device="cuda"), xf)
    xf = xf.cpu().numpy()
    val, _ = fe.tensor_basis(k, 3, oxi)
    ref = np.einsum("pj,pjr->pr", val, xc[cnode[ocell]])
    assert np.max(np.abs(xf[free[sel]] - ref)) <= 1e-12 * np.max(np.abs(xf))


def test_restriction_is_transpose_of_prolongation(full):
    name, cfg, levels, H, node_of, nn, cons, pts = full
    nrhs = cfg["nrhs"]
    for fl in range(1, len(levels)):
        g = torch.Generator(device="cuda").manual_seed(fl)
        xc = torch.randn(H.rows(fl - 1), nrhs, dtype=torch.float64, device="cuda", generator=g)
        yf = torch.randn(H.rows(fl), nrhs, dtype=torch.float64, device="cuda", generator=g)
        cc = torch.tensor(H.constrained(fl - 1), device="cuda")
        fc = torch.tensor(H.constrained(fl), device="cuda")
        xc[cc] = 0.0
        yf[fc] = 0.0
        px = H.vector(fl, nrhs)
        H.prolongate(fl, xc, px)
        ry = H.vector(fl - 1, nrhs)
        H.restrict(fl, yf, ry)
        lhs = (px * yf).sum(0)
        rhs = (xc * ry).sum(0)
        scale = (px.abs() * yf.abs()).sum(0)
        assert torch.all((lhs - rhs).abs() <= 1e-13 * scale)


def test_pcg_true_residual_and_modes(full):
    from paper_2412_10910_gb300 import _abi
    name, cfg, levels, H, node_of, nn, cons, pts = full
    top = len(levels) - 1
    nrhs = cfg["nrhs"]
    b = H.vector(top, nrhs)
    H.load_vector(top, np.ones(1), b, col=0)
    g = torch.Generator(device="cuda").manual_seed(3)
    b[:, 1:] = torch.randn(b.shape[0], nrhs - 1, dtype=torch.float64, device="cuda", generator=g)
    b[torch.tensor(cons, device="cuda")] = 0.0
    x32 = H.vector(top, nrhs)
    st, its, rel = H.pcg(b, x32, mode=_abi.FP32_MG_FP64_CG, rtol=1e-8, maxit=100)
    assert st == 0 and np.all(rel <= 1e-8)
    Ax = torch.empty_like(x32)
    H.apply(top, x32, Ax)
    true = ((b - Ax).norm(dim=0) / b.norm(dim=0)).cpu().numpy()
    assert np.all(true <= 2e-8), true
    x64 = H.vector(top, nrhs)
    st, its64, rel64 = H.pcg(b, x64, mode=_abi.FP64_MG, rtol=1e-8, maxit=100)
    assert st == 0 and np.all(np.abs(its64 - its) <= 1)
    err = ((x32 - x64).norm(dim=0) / x64.norm(dim=0)).cpu().numpy()
    assert np.all(err <= 1e-7), err
