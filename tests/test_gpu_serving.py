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
