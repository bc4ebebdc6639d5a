"""Seeded serving workload: 12 mesh families and a Poisson stream of solve requests.

Families (seed 5): 60% 2D / 40% 3D; degree uniform in {1,..,4}; fine cells per
direction uniform in [20, 600] (2D) or [8, 60] (3D); 3-5 levels with
n_{l-1} = floor((n_l - 1) / 2.2); interior jitter +-0.15h; further coarser
levels are added while the coarsest level has more than `coarse_cap` free
nodes.  Requests (seed 6): family uniform, 1-16 right-hand sides, N(0,1)
entries (seed 10000 + request id), exponential inter-arrival times.
"""
import numpy as np

from .meshes import _level


def serving_families(n_families=12, seed=5, coarse_cap=2000):
    rng = np.random.default_rng(seed)
    fams = []
    for f in range(n_families):
        dim = 2 if rng.random() < 0.6 else 3
        k = int(rng.integers(1, 5))
        n = int(rng.integers(20, 601)) if dim == 2 else int(rng.integers(8, 61))
        nl = int(rng.integers(3, 6))
        ns = [n]
        while ns[-1] > 1 and (len(ns) < nl or (k * ns[-1] - 1) ** dim > coarse_cap):
            ns.append(max(1, int((ns[-1] - 1) // 2.2)))
        ns = ns[::-1]
        levels = [_level((m,) * dim, (1.0,) * dim, 0.15, 1000 * (f + 1) + i)
                  for i, m in enumerate(ns)]
        fams.append(dict(name=f"fam{f:02d}_{dim}d_q{k}_n{n}", dim=dim, degree=k, levels=levels,
                         n_nodes=(k * n + 1) ** dim, n_free=(k * n - 1) ** dim))
    return fams


def serving_requests(families, n_requests=2000, seed=6, rate=1.0):
    """(family index, nrhs, arrival seconds) per request; arrivals at `rate` per second."""
    rng = np.random.default_rng(seed)
    fam = rng.integers(0, len(families), size=n_requests)
    nrhs = rng.integers(1, 17, size=n_requests)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    return [(int(f), int(m), float(t)) for f, m, t in zip(fam, nrhs, np.cumsum(gaps))]


def request_rhs(n_rows, nrhs, rid):
    return np.random.default_rng(10000 + rid).standard_normal((n_rows, nrhs))
