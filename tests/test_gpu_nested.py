"""Nested (global-coarsening) transfer: on nested meshes the sum-factorized
injection must equal the non-nested point evaluation (the same operator P,
Sec. 4.1) and the oracle's P; the V-cycle and PCG then agree as well."""
import numpy as np
import pytest

from synthetic.meshes import refine_nested
from tests.oracle_meshes import box_level

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _nested(dim, n0, n_ref, alpha=0.2, seed=3):
    lv = [box_level((n0,) * dim, alpha=alpha, seed=seed)]
    par = [None]
    for _ in range(n_ref):
        f, p, c = refine_nested(lv[-1])
        lv.append(f)
        par.append((p, c))
    return lv, par


@pytest.mark.parametrize("dim,k,nrhs", [(2, 3, 3), (3, 2, 8), (3, 4, 2)])
def test_nested_transfer_equals_point_evaluation_and_oracle(dim, k, nrhs):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.hierarchy import OracleHierarchy
    from paper_2412_10910_gb300 import nnmg
    lv, par = _nested(dim, 2 if dim == 3 else 3, 2)
    O = OracleHierarchy(lv, k, cheb_degree=3)
    H = nnmg.Hierarchy(lv, k, cheb_degree=3, max_nrhs=16)
    rng = np.random.default_rng(k)
    for l in range(1, len(lv)):
        xc = rng.standard_normal((O.levels[l - 1].n, nrhs))
        xc[O.levels[l - 1].constrained] = 0.0
        rf = rng.standard_normal((O.levels[l].n, nrhs))
        rf[O.levels[l].constrained] = 0.0
        for dt, tol in [(torch.float64, 1e-12), (torch.float32, 2e-5)]:
            out = {}
            for mode in ("nn", "gc"):
                H.set_nested(l, *(par[l] if mode == "gc" else (None, None)))
                xf = H.vector(l, nrhs, dt)
                H.prolongate(l, torch.tensor(xc, dtype=dt, device="cuda"), xf)
                rc = H.vector(l - 1, nrhs, dt)
                H.restrict(l, torch.tensor(rf, dtype=dt, device="cuda"), rc)
                out[mode] = (xf.double().cpu().numpy(), rc.double().cpu().numpy())
            po, ro = O.prolongate(l, xc), O.restrict(l, rf)
            for mode in ("nn", "gc"):
                assert np.max(np.abs(out[mode][0] - po)) <= tol * np.max(np.abs(po))
                assert np.max(np.abs(out[mode][1] - ro)) <= tol * np.max(np.abs(ro))
    # PCG with every level pair nested: same counts as the non-nested transfer
    top = len(lv) - 1
    b = H.vector(top, nrhs)
    b.normal_(generator=torch.Generator(device="cuda").manual_seed(5))
    b[torch.tensor(O.levels[top].constrained, device="cuda")] = 0.0
    x_gc, x_nn = H.vector(top, nrhs), H.vector(top, nrhs)
    for l in range(1, len(lv)):
        H.set_nested(l, *par[l])
    _, its_gc, rel_gc = H.pcg(b, x_gc)
    for l in range(1, len(lv)):
        H.set_nested(l)
    _, its_nn, rel_nn = H.pcg(b, x_nn)
    assert np.all(np.abs(its_gc - its_nn) <= 1) and np.all(rel_gc <= 1e-8)
    assert torch.max(torch.abs(x_gc - x_nn)) <= 1e-7 * torch.max(torch.abs(x_nn))
    H.close()


def test_set_nested_rejects_non_refinements():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import nnmg, _abi
    lv, par = _nested(2, 3, 1)
    H = nnmg.Hierarchy(lv, 2)
    p, c = par[1]
    c2 = c.copy()
    c2[0] = c2[1]                                   # two children at the same position
    with pytest.raises(nnmg.NNMGError) as e:
        H.set_nested(1, p, c2)
    assert e.value.status == _abi.INVALID_ARG
    H.close()
