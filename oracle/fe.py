"""1D bases, quadrature and the multilinear cell map, in plain FP64.

* Support points are the Gauss-Lobatto points on [0, 1] (Sec. 3.2, figure of
  the Gauss-Lobatto points for p = 4): the end points plus the roots of P_k'.
* Quadrature is Gauss-Legendre with k+1 points per direction (Sec. 4).
* The reference cell is [0, 1]^d (Sec. 3) and the geometry is the Q1 map from
  the 2^d cell vertices.
"""
import math
import numpy as np


def gauss_lobatto_nodes(k: int) -> np.ndarray:
    """k+1 Gauss-Lobatto nodes on [0,1] in closed form, k = 1..4."""
    if k == 1:
        return np.array([0.0, 1.0])
    if k == 2:
        return np.array([0.0, 0.5, 1.0])
    if k == 3:
        a = math.sqrt(5.0) / 10.0          # roots of P_3' are +-1/sqrt(5) on [-1,1]
        return np.array([0.0, 0.5 - a, 0.5 + a, 1.0])
    if k == 4:
        a = math.sqrt(21.0) / 14.0         # roots of P_4' are 0, +-sqrt(3/7)
        return np.array([0.0, 0.5 - a, 0.5, 0.5 + a, 1.0])
    raise ValueError("degree must be 1..4")


def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes and weights on [0,1] in closed form, n = 1..5."""
    if n == 1:
        t, w = [0.0], [2.0]
    elif n == 2:
        s = 1.0 / math.sqrt(3.0)
        t, w = [-s, s], [1.0, 1.0]
    elif n == 3:
        s = math.sqrt(0.6)
        t, w = [-s, 0.0, s], [5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0]
    elif n == 4:
        a = math.sqrt(3.0 / 7.0 - 2.0 / 7.0 * math.sqrt(6.0 / 5.0))
        b = math.sqrt(3.0 / 7.0 + 2.0 / 7.0 * math.sqrt(6.0 / 5.0))
        wa = (18.0 + math.sqrt(30.0)) / 36.0
        wb = (18.0 - math.sqrt(30.0)) / 36.0
        t, w = [-b, -a, a, b], [wb, wa, wa, wb]
    elif n == 5:
        a = math.sqrt(5.0 - 2.0 * math.sqrt(10.0 / 7.0)) / 3.0
        b = math.sqrt(5.0 + 2.0 * math.sqrt(10.0 / 7.0)) / 3.0
        wa = (322.0 + 13.0 * math.sqrt(70.0)) / 900.0
        wb = (322.0 - 13.0 * math.sqrt(70.0)) / 900.0
        t, w = [-b, -a, 0.0, a, b], [wb, wa, 128.0 / 225.0, wa, wb]
    else:
        raise ValueError("n must be 1..5")
    t = np.array(t)
    return 0.5 * (t + 1.0), 0.5 * np.array(w)


def lagrange(nodes: np.ndarray, x: np.ndarray):
    """Values and first derivatives of the Lagrange polynomials on `nodes`.

    Returns (L, dL) of shape [len(x), len(nodes)], from the product formula
    L_i(x) = prod_{m != i} (x - x_m) / (x_i - x_m) and its product-rule derivative.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    dL = np.zeros((len(x), n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            L[:, i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for q in range(n):
                if q == i or q == m:
                    continue
                term = term * (x - nodes[q]) / (nodes[i] - nodes[q])
            dL[:, i] += term
    return L, dL


def multi_indices(n: int, dim: int) -> np.ndarray:
    """Lexicographic multi-indices (x fastest) of an n^dim tensor grid: [n^dim, dim]."""
    idx = np.arange(n ** dim)
    return np.stack([(idx // n ** d) % n for d in range(dim)], axis=1)


def tensor_basis(k: int, dim: int, pts: np.ndarray):
    """Q_k basis values [P, nloc] and reference gradients [P, nloc, dim] at points [P, dim]."""
    nodes = gauss_lobatto_nodes(k)
    mi = multi_indices(k + 1, dim)
    tabs = [lagrange(nodes, pts[:, d]) for d in range(dim)]
    P = pts.shape[0]
    val = np.ones((P, len(mi)))
    grad = np.ones((P, len(mi), dim))
    for d in range(dim):
        Ld, dLd = tabs[d]
        val *= Ld[:, mi[:, d]]
        for a in range(dim):
            grad[:, :, a] *= (dLd if a == d else Ld)[:, mi[:, d]]
    return val, grad


def tensor_quadrature(n: int, dim: int):
    """Tensor Gauss-Legendre points [n^dim, dim] and weights [n^dim] on [0,1]^dim."""
    x, w = gauss_legendre(n)
    mi = multi_indices(n, dim)
    pts = x[mi]
    wts = np.prod(w[mi], axis=1)
    return pts, wts


def q1_shape(dim: int, xi: np.ndarray):
    """Q1 corner shape values [P, 2^d] and gradients [P, 2^d, d] at reference points [P, d]."""
    P = xi.shape[0]
    nv = 2 ** dim
    N = np.ones((P, nv))
    dN = np.ones((P, nv, dim))
    for v in range(nv):
        for d in range(dim):
            bit = (v >> d) & 1
            f = xi[:, d] if bit else 1.0 - xi[:, d]
            df = 1.0 if bit else -1.0
            N[:, v] *= f
            for a in range(dim):
                dN[:, v, a] *= (df if a == d else f)
    return N, dN
