"""Every operator kernel variant against the FP64 oracle.

The autotuner picks among the register-resident kernel (-1), its paired FP32
form (-2, two right-hand sides per thread in packed FP32 instructions), the
shared-memory kernel (units > 0; an unusable unit count keeps the default
block) and its paired FP32 form for 3D Poisson (-100 - U: U (cell, pair)
units per block; an odd nrhs, 2D levels and the other arithmetic types take
the default); NNMG_OP_CHOICE pins one choice for a whole hierarchy, so each variant
is checked on every level here whatever the timings would pick.  Tolerances
as in test_gpu_parity.py.
"""
import numpy as np
import pytest

from tests.gpu_cases import CASES, gpu_case, oracle_case, rng_vec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# cases with register-eligible levels: 2D Q1-Q4, 3D Q1-Q2, odd and even nrhs
NAMES = ["c1_q1", "c1_q3", "c1_q2_16rhs", "c1_q4_5rhs", "c2_q1_3lev", "c2_q2_3lev", "c3_q4_pmg"]
CHOICES = {"register": -1, "paired": -2, "shared": 1000000, "shared_paired": -108}
TOL = {"f64": 1e-12, "f32": 2e-5, "dw": 1e-12}


def _relmax(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module", params=NAMES)
def oracle(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    levels, O = oracle_case(request.param)
    return request.param, levels, O


@pytest.mark.parametrize("choice", list(CHOICES))
@pytest.mark.parametrize("dtype", ["f64", "f32", "dw"])
def test_operator_variant(oracle, choice, dtype, monkeypatch):
    name, levels, O = oracle
    monkeypatch.setenv("NNMG_OP_CHOICE", str(CHOICES[choice]))
    H = gpu_case(name, levels)
    try:
        nrhs = CASES[name][5]
        tdt = torch.float32 if dtype == "f32" else torch.float64
        for l in range(len(O.levels)):
            x = rng_vec(O.levels[l].n, nrhs, 40 + l)
            xo = x.copy()
            xo[np.repeat(O.levels[l].constrained, O.ncomp)] = 0.0
            yo = O.apply(l, xo)
            for _ in range(2):                 # the second call reuses the cached choice
                xt = torch.tensor(x, dtype=tdt, device="cuda")
                y = torch.full_like(xt, 3.0)
                H.apply(l, xt, y, double_word=(dtype == "dw"))
                err = _relmax(y.double().cpu().numpy(), yo)
                assert err <= TOL[dtype], (l, err)
    finally:
        H.close()


@pytest.mark.parametrize("choice", ["paired", "shared_paired"])
def test_paired_kernel_falls_back_on_unaligned_vectors(choice, monkeypatch):
    """The paired kernels read float pairs; vectors that start 4 bytes off an
    8-byte boundary must go to an unpaired kernel and give the same result."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    name = "c2_q2_3lev"
    levels, O = oracle_case(name)
    monkeypatch.setenv("NNMG_OP_CHOICE", str(CHOICES[choice]))
    H = gpu_case(name, levels)
    try:
        nrhs = CASES[name][5]
        top = len(O.levels) - 1
        n = O.levels[top].n * nrhs
        x = rng_vec(O.levels[top].n, nrhs, 77)
        xo = x.copy()
        xo[O.levels[top].constrained] = 0.0
        yo = O.apply(top, xo)
        xb = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
        yb = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
        xt = xb[1:].view(-1, nrhs)
        yt = yb[1:].view(-1, nrhs)
        assert xt.data_ptr() % 8 == 4 and yt.data_ptr() % 8 == 4
        xt.copy_(torch.tensor(x, dtype=torch.float32))
        H.apply(top, xt, yt)
        assert _relmax(yt.double().cpu().numpy(), yo) <= TOL["f32"]
        ya = torch.empty_like(xt.contiguous())
        H.apply(top, xt.clone(), ya)           # aligned: the paired kernel
        assert _relmax(ya.double().cpu().numpy(), yo) <= TOL["f32"]
    finally:
        H.close()


@pytest.mark.parametrize("choice", ["register", "paired", "shared_paired"])
def test_vcycle_and_pcg_with_variant(choice, monkeypatch):
    """The captured V-cycle and PCG graphs with a pinned kernel variant."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import _abi
    name = "c2_q2_3lev"
    levels, O = oracle_case(name)
    monkeypatch.setenv("NNMG_OP_CHOICE", str(CHOICES[choice]))
    H = gpu_case(name, levels)
    try:
        nrhs = CASES[name][5]
        top = len(O.levels) - 1
        b = rng_vec(O.levels[top].n, nrhs, 5)
        b[O.levels[top].constrained] = 0.0
        xo64, _, _, _ = O.pcg(b, "fp64", rtol=1e-8)
        _, its_o, _, _ = O.pcg(b, "fp32", rtol=1e-8)
        bt = torch.tensor(b, device="cuda")
        x = H.vector(top, nrhs)
        for _ in range(3):                      # eager, captured, replayed
            st, its, rel = H.pcg(bt, x, mode=_abi.FP32_MG_FP64_CG, rtol=1e-8, maxit=100)
            assert st == 0 and np.all(rel <= 1e-8)
            assert np.all(np.abs(its - np.array(its_o)) <= 1), (its, its_o)
            xs = x.cpu().numpy()
            err = np.linalg.norm(xs - xo64, axis=0) / np.linalg.norm(xo64, axis=0)
            assert np.all(err <= 1e-7), err
    finally:
        H.close()


def test_operator_choice_and_setup_phases_are_reported(monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import time
    from paper_2412_10910_gb300 import _abi, nnmg
    name = "c2_q2_3lev"
    levels, O = oracle_case(name)
    monkeypatch.setenv("NNMG_OP_CHOICE", "-1")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H = gpu_case(name, levels)
    wall = time.perf_counter() - t0
    try:
        phases = H.setup_seconds()
        assert list(phases) == list(nnmg.SETUP_PHASES)
        assert all(v >= 0.0 for v in phases.values())
        assert 0.0 < sum(phases.values()) <= wall
        nrhs = CASES[name][5]
        top = len(O.levels) - 1
        assert H.operator_choice(top, _abi.F64, nrhs) == 0          # not used yet
        x = torch.zeros(H.rows(top), nrhs, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        H.apply(top, x, y)
        assert H.operator_choice(top, _abi.F64, nrhs) == -1
        for bad in [(top + 1, _abi.F64, nrhs), (top, 7, nrhs), (top, _abi.F64, 0), (-1, _abi.F64, 1)]:
            with pytest.raises(nnmg.NNMGError):
                H.operator_choice(*bad)
    finally:
        H.close()


@pytest.mark.parametrize("name", ["c1_q1", "c1_q2_16rhs", "c2_q2_3lev", "c3_q4_pmg"])
def test_vcycle_and_pcg_with_and_without_persistent_smoother(name, monkeypatch):
    """The persistent smoother (one cooperative kernel per Chebyshev sweep on
    levels served by the register operator) and the kernel-per-step sequence
    give the same V-cycle and PCG: both against the oracle at the parity
    tolerances, and the same iteration counts."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import _abi
    levels, O = oracle_case(name)
    nrhs = CASES[name][5]
    top = len(O.levels) - 1
    r = rng_vec(O.levels[top].n, nrhs, 41)
    r[np.repeat(O.levels[top].constrained, O.ncomp)] = 0.0
    zo = O.vcycle(r, "fp64")
    r32 = torch.tensor(r, dtype=torch.float32, device="cuda")
    zo32 = O.vcycle(r32.double().cpu().numpy(), "fp32")
    its = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("NNMG_FUSED_SMOOTHER", fused)
        H = gpu_case(name, levels)
        try:
            for rep in range(2):               # eager, then the captured graph
                z = H.vector(top, nrhs)
                H.vcycle(torch.tensor(r, device="cuda"), z)
                assert _relmax(z.cpu().numpy(), zo) <= 1e-9, (fused, rep)
                z32 = H.vector(top, nrhs, torch.float32)
                H.vcycle(r32, z32)
                assert _relmax(z32.double().cpu().numpy(), zo32) <= 2e-5, (fused, rep)
            b = torch.tensor(r, device="cuda")
            x = H.vector(top, nrhs)
            st, it, rel = H.pcg(b, x, mode=_abi.FP32_MG_FP64_CG, rtol=1e-8, maxit=100)
            assert st == 0 and np.all(rel <= 1e-8)
            its[fused] = list(it)
        finally:
            H.close()
    assert its["1"] == its["0"]


@pytest.mark.parametrize("name", ["c1_q3", "c1_q4_5rhs", "c1_q2_16rhs", "c2_q2_3lev", "c3_q4_pmg"])
def test_fused_chebyshev_step_on_and_off(name, monkeypatch):
    """The Chebyshev steps as one operator + update launch (NNMG_FUSED_STEP=1)
    and as separate operator and vector kernels (the default): V-cycles in
    FP64 and FP32 against the oracle's, repeated (the per-node counts must be
    back at zero after every step), and against each other."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    levels, O = oracle_case(name)
    nrhs = CASES[name][5]
    top = len(O.levels) - 1
    r = rng_vec(O.levels[top].n, nrhs, 41)
    r[np.repeat(O.levels[top].constrained, O.ncomp)] = 0.0
    zo = O.vcycle(r, "fp64")
    zo32 = O.vcycle(r.astype(np.float32).astype(np.float64), "fp32")
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("NNMG_FUSED_STEP", flag)
        H = gpu_case(name, levels)
        try:
            for _ in range(3):                                 # eager, captured, replayed
                z = H.vector(top, nrhs)
                H.vcycle(torch.tensor(r, device="cuda"), z)
                assert _relmax(z.cpu().numpy(), zo) <= 1e-9, flag
                z32 = H.vector(top, nrhs, torch.float32)
                H.vcycle(torch.tensor(r, dtype=torch.float32, device="cuda"), z32)
                assert _relmax(z32.double().cpu().numpy(), zo32) <= 2e-5, flag
            out[flag] = z.cpu().numpy()
        finally:
            H.close()
    assert _relmax(out["1"], out["0"]) <= 1e-12
