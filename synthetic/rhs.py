"""Random right-hand sides: one numpy Generator per column, N(0, 1)."""
import numpy as np


def normal_rhs(n_rows: int, seeds) -> np.ndarray:
    """[n_rows, len(seeds)] float64; column j drawn from default_rng(seeds[j])."""
    cols = [np.random.default_rng(int(s)).standard_normal(n_rows) for s in seeds]
    return np.ascontiguousarray(np.stack(cols, axis=1))
