"""Continuous batching: requests that arrive while others are solved join the
running PCG of their family; each result must be the same alone and in the
mix (relative L2 difference <= 1e-9, iteration counts within +-1, relative
residual <= 1e-8), also when the memory budget forces families out."""
import numpy as np
import pytest

from synthetic.meshes import config_levels, family_levels

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _families():
    from paper_2412_10910_gb300.serving import FamilySpec
    return {
        "2d_q2": FamilySpec(config_levels("c1_2d_q1"), 2),
        "3d_q1": FamilySpec(family_levels(3, 19, 3, 0.15, 40), 1),
        "2d_q3": FamilySpec(family_levels(2, 30, 3, 0.15, 50), 3),
    }


def _requests(server, n=14, seed=0):
    from paper_2412_10910_gb300.serving import Request
    rng = np.random.default_rng(seed)
    names = sorted(server.families)
    reqs = []
    for i in range(n):
        fam = names[rng.integers(len(names))]
        eng = server.engine(fam)
        cons = np.repeat(eng.H.constrained(eng.top), 1)
        nrhs = int(rng.integers(1, 7))
        b = rng.standard_normal((eng.rows, nrhs))
        b[cons] = 0.0
        reqs.append(Request(i, fam, b, arrival=0.002 * i))
    return reqs


def _alone(families, req):
    from paper_2412_10910_gb300 import nnmg
    spec = families[req.family]
    H = nnmg.Hierarchy(spec.levels, spec.degree, cheb_degree=spec.cheb, max_nrhs=16)
    b = torch.tensor(req.b, device="cuda")
    x = torch.zeros_like(b)
    st, its, rel = H.pcg(b, x)
    out = x.cpu().numpy(), its
    H.close()
    return out


@pytest.mark.parametrize("budget_gb", [64.0, None])
def test_each_result_same_alone_and_in_the_mix(budget_gb):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300.serving import Server, latency_stats
    fams = _families()
    probe = Server(fams, budget_bytes=1 << 40)
    sizes = {n: probe.engine(n).bytes() for n in fams}
    reqs = _requests(probe)
    probe.close()
    # budget None: room for the largest family plus a little, forcing evictions
    budget = int(budget_gb * 2 ** 30) if budget_gb else int(max(sizes.values()) * 1.5)
    server = Server(fams, budget_bytes=budget)
    done = server.run(reqs)
    assert len(done) == len(reqs)
    if budget_gb is None:
        assert server.evictions > 0
    else:                                   # the batches changed width on the way
        assert sum(e.repacks for e in server.engines.values()) > 0
    for r in done:
        assert all(s == 0 for s in r.status) and max(r.relres) <= 1e-8
        xa, its = _alone(fams, r)
        err = np.linalg.norm(r.x - xa, axis=0) / np.linalg.norm(xa, axis=0)
        assert np.all(err <= 1e-9), (r.rid, err)
        assert np.all(np.abs(np.array(r.iters) - its) <= 1)
    st = latency_stats(done)
    assert st["p99_s"] >= st["p50_s"] > 0
    server.close()


def test_size_estimate_equals_built_bytes():
    """nnmg_estimate_bytes (host only, before setup) equals what the built
    hierarchy reports, for Poisson, elasticity and polynomial-coarsening
    hierarchies."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300 import nnmg
    cases = [(config_levels("c1_2d_q1"), 2, 1, None),
             (family_levels(3, 19, 3, 0.15, 40), 1, 1, None),
             (config_levels("c4_3d_q2_elasticity", n_levels=2), 2, 3, None),
             ([config_levels("c2_3d_q2", n_levels=1)[0]] + config_levels("c2_3d_q2", n_levels=2),
              2, 1, [1, 2, 2])]
    for levels, k, nc, degs in cases:
        for nrhs in (1, 16):
            hb, sb = nnmg.nnmg_estimate_bytes(levels, k, nc, nrhs=nrhs, level_degrees=degs)
            H = nnmg.Hierarchy(levels, k, nc, level_degrees=degs)
            assert (hb, sb) == (H.hierarchy_bytes(), H.solve_bytes(nrhs))
            H.close()


def test_a_waiting_family_allocates_nothing():
    """Budget for one family at a time, the built one busy: the other family
    waits, is not built, and device free memory does not change."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_10910_gb300.serving import FamilyEngine, Server
    fams = _families()
    sizes = {n: FamilyEngine.estimate_bytes(n, s) for n, s in fams.items()}
    a, b = sorted(sizes, key=sizes.get)[:2]
    server = Server(fams, budget_bytes=sizes[a] + sizes[b] - 1)
    ea = server.engine(a)
    ea.queue.append(None)                     # a queued request keeps it busy
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert server.engine(b) is None
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert server.builds == 1 and list(server.engines) == [a]
    ea.queue.clear()
    assert server.engine(b) is not None and server.evictions == 1
    server.close()


def test_repack_continues_every_column():
    """nnmg_batch_repack between steps: narrowing with a permutation that
    drops columns, then widening and admitting into new columns (one column
    from the device, two from a host block with nnmg_batch_admit_cols); every
    continued column ends as its solve alone (relative L2 difference <= 1e-9,
    iterations +-1).  Maps with repeated or out-of-range slots, widths outside
    1..max_nrhs, a repack while a step is in flight and column blocks outside
    the batch or with a bad leading dimension are rejected."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes as C
    from paper_2412_10910_gb300 import _abi, nnmg
    spec = _families()["2d_q3"]
    H = nnmg.Hierarchy(spec.levels, spec.degree, cheb_degree=spec.cheb, max_nrhs=16)
    lib = _abi.load()
    top = H.n_levels - 1
    rows = H.rows(top)
    sp = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(3)
    B = rng.standard_normal((rows, 7))
    B[H.constrained(top)] = 0.0
    bt = torch.tensor(B.T.copy(), device="cuda")          # bt[j] = column j
    n = 16
    active = np.zeros(n, dtype=np.int32)
    iters = np.zeros(n, dtype=np.int32)
    rel = np.zeros(n)
    status = np.zeros(n, dtype=np.int32)

    def ok(rc):
        assert rc == _abi.OK, lib.nnmg_last_error()

    def repack(src, width=None):
        width = len(src) if width is None else width
        return lib.nnmg_batch_repack(H.h, width, (C.c_int * max(1, len(src)))(*src), sp)

    def step_and_poll(k):
        ok(lib.nnmg_batch_step(H.h, k, sp))
        ready = C.c_int(0)
        ok(lib.nnmg_batch_poll(H.h, 1, C.byref(ready), active.ctypes.data, iters.ctypes.data,
                               rel.ctypes.data, status.ctypes.data))
        assert ready.value == 1

    try:
        ok(lib.nnmg_batch_reset(H.h, _abi.FP32_MG_FP64_CG, n, 1e-8, 200, sp))
        for j in range(6):
            ok(lib.nnmg_batch_admit(H.h, j, C.c_void_p(bt[j].data_ptr()), 0, sp))
        step_and_poll(2)
        assert np.all(active[:6] == 1)
        # rejected maps: repeated slot, slot beyond the batch, widths 0 and 17
        for src, width in (([0, 0], None), ([16], None), ([0], 0), (list(range(16)) + [-1], 17)):
            assert repack(src, width) == _abi.INVALID_ARG
        ok(lib.nnmg_batch_step(H.h, 1, sp))              # a step in flight
        assert repack([0, 1]) == _abi.INVALID_ARG
        ready = C.c_int(0)
        ok(lib.nnmg_batch_poll(H.h, 1, C.byref(ready), None, None, None, None))
        # narrow to 4 columns: old 5, 2, empty, old 0 (old 1, 3, 4 dropped)
        ok(repack([5, 2, -1, 0]))
        step_and_poll(2)
        assert list(active[:4]) == [1, 1, 0, 1]
        # widen to 6 columns: the three running ones, a new right-hand side in
        # column 2 and, from a host block [rows][3], two more in columns 4-5
        ok(repack([0, 1, -1, 3, -1, -1]))
        ok(lib.nnmg_batch_admit(H.h, 2, C.c_void_p(bt[6].data_ptr()), 0, sp))
        blk = np.ascontiguousarray(B[:, [1, 3, 4]])
        for first, ncols, ldb in ((5, 2, 3), (4, 3, 2), (4, 2, 17)):
            assert lib.nnmg_batch_admit_cols(H.h, first, ncols, blk.ctypes.data, ldb, 1, sp) == \
                _abi.INVALID_ARG
        ok(lib.nnmg_batch_admit_cols(H.h, 4, 2, blk.ctypes.data, 3, 1, sp))
        for _ in range(200):
            step_and_poll(1)
            if not np.any(active[:6]):
                break
        assert np.all(status[:6] == 0) and np.all(rel[:6] <= 1e-8)
        got = {}
        for slot, col in ((0, 5), (1, 2), (2, 6), (3, 0), (4, 1), (5, 3)):
            xs = torch.empty(rows, dtype=torch.float64, device="cuda")
            ok(lib.nnmg_batch_retire(H.h, slot, C.c_void_p(xs.data_ptr()), 0, sp))
            torch.cuda.synchronize()
            got[col] = (xs.cpu().numpy(), int(iters[slot]))
        for col, (xg, it) in got.items():
            b1 = torch.tensor(B[:, col:col + 1], device="cuda")
            x1 = torch.zeros_like(b1)
            st, its, _ = H.pcg(b1, x1)
            xa = x1.cpu().numpy()[:, 0]
            assert np.linalg.norm(xg - xa) <= 1e-9 * np.linalg.norm(xa), col
            assert abs(it - int(its[0])) <= 1, (col, it, its)
    finally:
        H.close()
