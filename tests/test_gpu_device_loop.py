"""The device-side PCG loop (a CUDA graph WHILE node around one iteration)
against the host-driven loop and the oracle.

Both loops replay the same captured iteration, so they agree to the rounding
of the operator's floating-point atomics (relative 1e-12, identical iteration
counts); the solution is held to the oracle as in test_gpu_parity.py.  Edge
cases: a zero right-hand side (no iteration runs), maxit reached (the loop's
own cap ends it), and a transfer change (nnmg_set_nested) that must rebuild
the loop.
"""
import numpy as np
import pytest

from tests.gpu_cases import CASES, gpu_case, oracle_case, rng_vec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solve(H, b, mode, reps, **kw):
    top = H.n_levels - 1
    bt = torch.tensor(b, device="cuda")
    out = []
    for _ in range(reps):
        x = H.vector(top, b.shape[1])
        st, its, rel = H.pcg(bt, x, mode=mode, allow_fail=True, **kw)
        out.append((st, np.asarray(its).copy(), np.asarray(rel).copy(), x.cpu().numpy()))
    return out


@pytest.mark.parametrize("name", ["c1_q1", "c2_q2_3lev", "c4_elast", "c3_q4_pmg"])
@pytest.mark.parametrize("mode_name", ["fp32", "fp64", "dw"])
def test_device_loop_matches_host_loop_and_oracle(name, mode_name, monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import _abi
    mode = {"fp32": _abi.FP32_MG_FP64_CG, "fp64": _abi.FP64_MG, "dw": _abi.FP32_MG_DW_CG}[mode_name]
    levels, O = oracle_case(name)
    nrhs = CASES[name][5]
    top = len(O.levels) - 1
    b = rng_vec(O.levels[top].n, nrhs, 60)
    b[np.repeat(O.levels[top].constrained, O.ncomp)] = 0.0
    xo64, _, _, _ = O.pcg(b, "fp64", rtol=1e-8)
    monkeypatch.setenv("NNMG_DEVICE_LOOP", "0")
    Hh = gpu_case(name, levels)
    try:
        host = _solve(Hh, b, mode, 3)
        assert Hh.pcg_device_loop(mode, nrhs) == 0
    finally:
        Hh.close()
    monkeypatch.delenv("NNMG_DEVICE_LOOP")
    Hd = gpu_case(name, levels)
    try:
        dev = _solve(Hd, b, mode, 3)                  # eager, captured, device loop
        assert Hd.pcg_device_loop(mode, nrhs) == 1
    finally:
        Hd.close()
    st_h, its_h, rel_h, x_h = host[-1]
    for st, its, rel, x in dev:
        assert st == 0 and st_h == 0
        np.testing.assert_array_equal(its, its_h)
        assert np.all(rel <= 1e-8)
        assert np.max(np.abs(x - x_h)) <= 1e-12 * np.max(np.abs(x_h))
        err = np.linalg.norm(x - xo64, axis=0) / np.linalg.norm(xo64, axis=0)
        assert np.all(err <= 1e-7), err


def test_device_loop_zero_rhs_and_maxit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import _abi
    name = "c2_q2_3lev"
    levels, O = oracle_case(name)
    nrhs = CASES[name][5]
    top = len(O.levels) - 1
    H = gpu_case(name, levels)
    try:
        b = rng_vec(O.levels[top].n, nrhs, 61)
        b[O.levels[top].constrained] = 0.0
        b[:, 3] = 0.0                                  # one column without work
        mode = _abi.FP32_MG_FP64_CG
        runs = _solve(H, b, mode, 3)
        assert H.pcg_device_loop(mode, nrhs) == 1
        for st, its, rel, x in runs:
            assert st == 0 and its[3] == 0 and np.all(x[:, 3] == 0.0)
        # maxit reached: the loop's own cap ends it, x is still written
        capped = _solve(H, b, mode, 2, rtol=1e-30, maxit=3)
        for st, its, rel, x in capped:
            assert st == _abi.NOT_CONVERGED
            assert np.all(its[np.arange(nrhs) != 3] == 3) and its[3] == 0
            assert np.all(np.isfinite(x))
        # all columns zero: no iteration at all
        z = _solve(H, np.zeros_like(b), mode, 2)
        for st, its, rel, x in z:
            assert st == 0 and np.all(its == 0) and np.all(x == 0.0)
    finally:
        H.close()


def test_device_loop_rebuilt_after_transfer_change():
    """nnmg_set_nested changes the V-cycle; a loop captured before must not be
    replayed after it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import _abi, nnmg
    from synthetic.meshes import refine_nested
    from tests.oracle_meshes import box_level
    coarse = box_level((2, 2, 2), alpha=0.2, seed=3)
    mid, p1, c1 = refine_nested(coarse)
    fine, p2, c2 = refine_nested(mid)
    levels = [coarse, mid, fine]
    mode = _abi.FP32_MG_FP64_CG
    H = nnmg.Hierarchy(levels, 2, 1, cheb_degree=3, max_nrhs=16)
    Hn = nnmg.Hierarchy(levels, 2, 1, cheb_degree=3, max_nrhs=16)
    try:
        Hn.set_nested(1, p1, c1)
        Hn.set_nested(2, p2, c2)
        top = H.n_levels - 1
        b = H.vector(top, 2)
        H.load_vector(top, np.ones(1), b, col=0)
        b[:, 1] = b[:, 0]
        bn = b.cpu().numpy()
        _solve(H, bn, mode, 3)
        assert H.pcg_device_loop(mode, 2) == 1
        H.set_nested(1, p1, c1)
        H.set_nested(2, p2, c2)
        assert H.pcg_device_loop(mode, 2) == 0          # dropped with the old V-cycle
        after = _solve(H, bn, mode, 3)
        ref = _solve(Hn, bn, mode, 3)
        for (st, its, rel, x), (st2, its2, rel2, x2) in zip(after, ref):
            assert st == 0 and st2 == 0
            np.testing.assert_array_equal(its, its2)
            assert np.max(np.abs(x - x2)) <= 1e-12 * np.max(np.abs(x2))
    finally:
        H.close()
        Hn.close()
