"""Full-size parity: configuration 2 (the benchmark's launch configuration:
3D Q2, 55^3 fine cells, 8 right-hand sides), configuration 3 (3D Q4 on the
deformed cube, 39^3 fine cells, 4 right-hand sides) and the throughput
hierarchy of configuration 4 (vector Q2 elasticity on the beam with a fourth,
85x23x23-cell level: 1,133,217 DoFs, 1 right-hand side).

At these sizes the oracle computes sampled outputs one by one: the DoF
numbering of the whole fine mesh, operator rows from the element matrices of
the cells around sampled nodes, located points and prolongated values at
sampled fine nodes.  Properties that hold at any size cover the rest:
<P x, y> = <x, P^T y> for restriction, symmetry and positivity of the whole
V-cycle (Algorithm 1 with Chebyshev smoothing is a symmetric positive definite
preconditioner), the agreement of its FP32 and FP64 runs, the true residual
of the PCG solution and the agreement of the two precision modes.  The
V-cycle itself is compared element by element with the oracle's on the three
coarsest levels of the configuration 2 family at the full 8 right-hand sides
(case c2_q2_3lev of test_gpu_parity.py: FP64 at 1e-9, FP32 at 2e-5 against
the oracle's float V-cycle).  Tolerances as in test_gpu_parity.py.
"""
import numpy as np
import pytest

from oracle import assembly, dofs, fe, transfer
from synthetic import config_levels
from synthetic.meshes import CONFIGS

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# name -> (configuration, cell counts per level or None for the stated ones)
FULL = {
    "c2_3d_q2": ("c2_3d_q2", None),
    "c3_3d_q4_deformed": ("c3_3d_q4_deformed", None),
    "c4_beam_85x23x23": ("c4_3d_q2_elasticity", [(8, 2, 2), (19, 5, 5), (41, 11, 11), (85, 23, 23)]),
}


@pytest.fixture(scope="module", params=list(FULL))
def full(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import nnmg
    name, cells = FULL[request.param]
    cfg = dict(CONFIGS[name])
    levels = config_levels(name, cells=cells)
    H = nnmg.Hierarchy(levels, cfg["degree"], cfg["ncomp"], cfg.get("lame", (1.0, 1.0)),
                       cheb_degree=cfg["cheb"], max_nrhs=16)
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
    nrhs, k, nc = cfg["nrhs"], cfg["degree"], cfg["ncomp"]
    rng = np.random.default_rng(7)
    x = rng.standard_normal((nn, nc, nrhs))
    x[cons] = 0.0
    tdt = torch.float64 if dtype == "f64" else torch.float32
    xt = torch.tensor(x.reshape(nn * nc, nrhs), dtype=tdt, device="cuda")
    y = torch.empty_like(xt)
    H.apply(top, xt, y)
    y = y.double().cpu().numpy().reshape(nn, nc, nrhs)
    xin = xt.double().cpu().numpy().reshape(nn, nc, nrhs)   # the exact input the kernel saw
    sample = rng.choice(np.nonzero(~cons)[0], 300, replace=False)
    cells = np.unique(np.nonzero(np.isin(node_of, sample))[0])
    E = assembly.element_matrices(f.vertices, f.cells[cells], k, 3, nc, cfg.get("lame", (1.0, 1.0)))
    yo = np.zeros((nn, nc, nrhs))
    nloc = node_of.shape[1]
    for c, Ec in zip(cells, E):
        loc = node_of[c]
        yo[loc] += (Ec @ xin[loc].reshape(nloc * nc, nrhs)).reshape(nloc, nc, nrhs)
    ref = yo[sample]
    scale = np.max(np.abs(y))
    assert np.max(np.abs(y[sample] - ref)) <= tol * scale
    assert np.all(y[cons] == 0.0)


def test_point_location_and_prolongation_sampled(full):
    name, cfg, levels, H, node_of, nn, cons, pts = full
    top = len(levels) - 1
    c = levels[top - 1]
    k, nrhs, nc = cfg["degree"], cfg["nrhs"], cfg["ncomp"]
    cnode, cnn, _, _ = dofs.number_dofs(c.cells, k, 3)
    ccons = dofs.dirichlet_nodes(c.cells, c.dirichlet, cnode, k, 3)
    cell, xi = H.transfer_points(top)
    free = np.nonzero(~cons)[0]
    rng = np.random.default_rng(11)
    sel = rng.choice(len(free), 300, replace=False)
    ocell, oxi = transfer.locate(pts[free[sel]], c.vertices, c.cells, 3)
    np.testing.assert_array_equal(cell[sel], ocell)
    np.testing.assert_allclose(xi[sel], oxi, rtol=0, atol=1e-12)
    for dtype, tol in (("f64", 1e-12), ("f32", 2e-5)):
        tdt = torch.float64 if dtype == "f64" else torch.float32
        xc = rng.standard_normal((cnn, nc, nrhs))
        xc[ccons] = 0.0
        xct = torch.tensor(xc.reshape(cnn * nc, nrhs), dtype=tdt, device="cuda")
        xf = H.vector(top, nrhs, tdt)
        H.prolongate(top, xct, xf)
        xf = xf.double().cpu().numpy().reshape(nn, nc, nrhs)
        xcin = xct.double().cpu().numpy().reshape(cnn, nc, nrhs)
        val, _ = fe.tensor_basis(k, 3, oxi)
        ref = np.einsum("pj,pjcr->pcr", val, xcin[cnode[ocell]])
        assert np.max(np.abs(xf[free[sel]] - ref)) <= tol * np.max(np.abs(xf)), dtype


def test_restriction_is_transpose_of_prolongation(full):
    name, cfg, levels, H, node_of, nn, cons, pts = full
    nrhs, nc = cfg["nrhs"], cfg["ncomp"]
    for fl in range(1, len(levels)):
        g = torch.Generator(device="cuda").manual_seed(fl)
        xc = torch.randn(H.rows(fl - 1), nrhs, dtype=torch.float64, device="cuda", generator=g)
        yf = torch.randn(H.rows(fl), nrhs, dtype=torch.float64, device="cuda", generator=g)
        cc = torch.tensor(np.repeat(H.constrained(fl - 1), nc), device="cuda")
        fc = torch.tensor(np.repeat(H.constrained(fl), nc), device="cuda")
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


def test_vcycle_symmetric_positive_and_precisions_agree(full):
    """The whole V-cycle at full size: <V r1, r2> = <r1, V r2> and <V r, r> > 0
    per column in FP64 (the oracle's V-cycle has these properties, pinned in
    test_oracle_solver.py), and the FP32 V-cycle equals the FP64 one within
    the FP32 tolerance."""
    name, cfg, levels, H, node_of, nn, cons, pts = full
    top = len(levels) - 1
    nrhs, nc = cfg["nrhs"], cfg["ncomp"]
    g = torch.Generator(device="cuda").manual_seed(5)
    fc = torch.tensor(np.repeat(cons, nc), device="cuda")
    r1 = torch.randn(H.rows(top), nrhs, dtype=torch.float64, device="cuda", generator=g)
    r2 = torch.randn(H.rows(top), nrhs, dtype=torch.float64, device="cuda", generator=g)
    r1[fc] = 0.0
    r2[fc] = 0.0
    z1, z2 = H.vector(top, nrhs), H.vector(top, nrhs)
    H.vcycle(r1, z1)
    H.vcycle(r2, z2)
    a, b = (z1 * r2).sum(0), (r1 * z2).sum(0)
    scale = (z1.abs() * r2.abs()).sum(0)
    assert torch.all((a - b).abs() <= 1e-12 * scale), ((a - b).abs() / scale).tolist()
    assert torch.all((z1 * r1).sum(0) > 0)
    z32 = H.vector(top, nrhs, torch.float32)
    H.vcycle(r1.float(), z32)
    rel = ((z32.double() - z1).abs().max() / z1.abs().max()).item()
    assert rel <= 2e-5, rel


def test_pcg_true_residual_and_modes(full):
    from paper_2412_10910_gb300 import _abi
    name, cfg, levels, H, node_of, nn, cons, pts = full
    top = len(levels) - 1
    nrhs, nc = cfg["nrhs"], cfg["ncomp"]
    b = H.vector(top, nrhs)
    # f = 1 (Poisson) or the beam's body load (0, 0, -1) in column 0
    H.load_vector(top, np.ones(1) if nc == 1 else np.array([0.0, 0.0, -1.0]), b, col=0)
    g = torch.Generator(device="cuda").manual_seed(3)
    if nrhs > 1:
        b[:, 1:] = torch.randn(b.shape[0], nrhs - 1, dtype=torch.float64, device="cuda", generator=g)
    b[torch.tensor(np.repeat(cons, nc), device="cuda")] = 0.0
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
