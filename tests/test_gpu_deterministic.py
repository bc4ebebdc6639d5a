"""Deterministic mode (nnmg_options.deterministic = 1): cells stored in
vertex-disjoint colors, one launch per color in every cell loop.  Checked:
the stored colors are valid and hold every cell once; operator, V-cycle and
PCG match the FP64 oracle at the tolerances of test_gpu_parity.py; repeated
operator applications, V-cycles and solves (eager, captured, replayed), and a
second hierarchy built from scratch, give bitwise identical results."""
import numpy as np
import pytest

from tests.gpu_cases import CASES, gpu_case, oracle_case, rng_vec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAMES = ["c2_q2_3lev", "c4_elast", "c1_q3", "c3_q4_pmg", "annulus_q2"]


def _relmax(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module", params=NAMES)
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    levels, O = oracle_case(request.param)
    H = gpu_case(request.param, levels, deterministic=True)
    yield request.param, levels, O, H
    H.close()


def test_colors_are_vertex_disjoint_and_cover_every_cell(case):
    from paper_2412_10910_gb300 import nnmg
    name, levels, O, H = case
    for l in range(H.n_levels):
        cs = nnmg.nnmg_level_colors(H.h, l)
        cn = H.cell_nodes(l)
        assert len(cs) >= 2 and cs[0] == 0 and cs[-1] == len(cn) and np.all(np.diff(cs) >= 0)
        # the input's cells regrouped, numbering unchanged: the same node rows
        assert sorted(map(tuple, cn)) == sorted(map(tuple, np.asarray(O.levels[l].node_of)))
        for c in range(len(cs) - 1):
            rows = cn[cs[c]:cs[c + 1]].ravel()
            assert len(np.unique(rows)) == len(rows), (l, c)      # no node shared within a color


def test_operator_matches_oracle_and_repeats_bitwise(case):
    name, levels, O, H = case
    nrhs = CASES[name][5]
    for l in range(len(O.levels)):
        x = rng_vec(O.levels[l].n, nrhs, 60 + l)
        xo = x.copy()
        xo[np.repeat(O.levels[l].constrained, O.ncomp)] = 0.0
        yo = O.apply(l, xo)
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
            xt = torch.tensor(x, dtype=dt, device="cuda")
            ys = []
            for _ in range(3):
                y = torch.zeros_like(xt)
                H.apply(l, xt, y)
                ys.append(y)
            assert _relmax(ys[0].double().cpu().numpy(), yo) <= tol
            assert all(torch.equal(ys[0], y) for y in ys[1:]), (l, dt)


def test_vcycle_and_pcg_match_oracle_and_repeat_bitwise(case):
    from paper_2412_10910_gb300 import _abi
    name, levels, O, H = case
    nrhs = CASES[name][5]
    top = len(O.levels) - 1
    r = rng_vec(O.levels[top].n, nrhs, 40)
    ro = r.copy()
    ro[np.repeat(O.levels[top].constrained, O.ncomp)] = 0.0
    zo = O.vcycle(ro, "fp64")
    zs = []
    for _ in range(3):                         # eager, captured, replayed
        z = H.vector(top, nrhs)
        H.vcycle(torch.tensor(r, device="cuda"), z)
        zs.append(z)
    assert _relmax(zs[0].cpu().numpy(), zo) <= 1e-9
    assert all(torch.equal(zs[0], z) for z in zs[1:])
    b = rng_vec(O.levels[top].n, nrhs, 50)
    b[np.repeat(O.levels[top].constrained, O.ncomp)] = 0.0
    xo64, _, _, _ = O.pcg(b, "fp64", rtol=1e-8)
    bt = torch.tensor(b, device="cuda")
    runs = []
    for _ in range(3):
        x = H.vector(top, nrhs)
        st, its, rel = H.pcg(bt, x, mode=_abi.FP32_MG_FP64_CG, rtol=1e-8)
        assert st == 0 and np.all(rel <= 1e-8)
        runs.append((x, list(its)))
    err = np.linalg.norm(runs[0][0].cpu().numpy() - xo64, axis=0) / np.linalg.norm(xo64, axis=0)
    assert np.all(err <= 1e-7), err
    assert all(torch.equal(runs[0][0], x) and its == runs[0][1] for x, its in runs[1:])
    # a second hierarchy built from the same levels: setup (diagonal, Lanczos,
    # coarse inverse) and solve repeat bitwise
    H2 = gpu_case(name, levels, deterministic=True)
    try:
        x2 = H2.vector(top, nrhs)
        st, its, rel = H2.pcg(bt, x2, mode=_abi.FP32_MG_FP64_CG, rtol=1e-8)
        assert torch.equal(runs[0][0], x2) and list(its) == runs[0][1]
    finally:
        H2.close()
