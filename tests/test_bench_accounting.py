"""Host logic of the measurement: the operation count that the roofline's
numerator uses and the algorithmic bytes of the fine-level kernel table.

The FP64 pipe operations per cell and right-hand side of the 3D Poisson
operator (bench.poisson3d_work) are recounted here by walking the sweeps the
register kernel runs, entry by entry, with the exact zeros it skips: for an
odd point count the interpolation matrix S has a unit middle row (the middle
Gauss point is the middle Lobatto node) and the collocation derivative Dg a
zero middle diagonal entry.  A product chain starts with a multiplication,
so a row of e nonzero entries costs e operations (2e - 1 flops), and an
accumulating row one more of each.
"""
import bench


def _apply_count(n, kind, transpose, add):
    """(ops, flops) of one line of M (transpose=False) or M^T (transpose=True,
    add=True accumulating into the line), M = S or Dg, as the kernel runs it."""
    odd = n % 2 == 1
    mid = n // 2

    def unit_row(q):
        return kind == "S" and odd and q == mid

    def zero(q, l):
        if not odd:
            return False
        return (q == mid and l != mid) if kind == "S" else (q == mid and l == mid)

    ops = flops = 0
    for out in range(n):
        if not transpose:
            if unit_row(out):
                continue                        # a copy
            first = True
            for l in range(n):
                if zero(out, l):
                    continue
                ops += 1
                flops += 1 if first else 2      # multiply, then multiply-adds
                first = False
            continue
        first = not add                         # accumulating: starts from the line
        if unit_row(out):                       # the unit entry M[out][out] = 1
            if not first:
                ops += 1
                flops += 1
            first = False
        for q in range(n):
            if zero(q, out) or unit_row(q):
                continue
            ops += 1
            flops += 1 if first else 2
            first = False
    return ops, flops


def _cell_count(n):
    lines = n * n
    ops = flops = 0
    for kind, transpose, add, sweeps in (("S", False, False, 3), ("D", False, False, 3),
                                         ("D", True, False, 1), ("D", True, True, 2),
                                         ("S", True, False, 3)):
        o, f = _apply_count(n, kind, transpose, add)
        ops += sweeps * lines * o
        flops += sweeps * lines * f
    q = n ** 3
    return flops + 15 * q, ops + 9 * q


def test_operator_operation_counts():
    for n in (2, 3, 4, 5):
        assert bench.poisson3d_work(n) == _cell_count(n), n
    # the values quoted with the roofline: Q2 and Q4
    assert bench.poisson3d_work(3) == (1701, 999)
    assert bench.poisson3d_work(5)[1] == 7725


def test_fine_level_kernel_bytes_by_hand():
    # a 2^3-cell Q1 level above a 1-cell Q1 level, 2 RHS, FP32, Chebyshev 3
    fine = (27, 1, 8)          # nodes, free nodes, cells
    coarse = (8, 0, 1)
    by = bench.fine_level_kernel_bytes(3, 1, 1, 1, 2, 4, 3, fine, coarse)
    # operator: x read + y write at the free row, metric 6 x 8 points x 4 B and
    # 8 indices per cell
    assert by["operator"] == 2 * 1 * 2 * 4 + 8 * 8 * (6 * 4 + 4)
    # vector kernels: 27 rows x 2 RHS x 4 B x (3 + 5 x 7) + 6 diagonal passes
    assert by["vector"] == 27 * 2 * 4 * (3 + 5 * 7) + 6 * 27 * 4
    pts = 1 * (4 + 3 * 4)
    buf = 1 * 8 * 2 * 4
    # fused residual: f and t read and t reset at the one located point
    assert by["restrictor"] == 3 * 1 * 2 * 4 + pts + 8 * 2 * 4 + 2 * buf + 8 * 4
    assert by["prolongator"] == 8 * 2 * 4 + 8 * 4 + 2 * 1 * 2 * 4 + pts
