"""Plain FP64 CPU oracle for the non-nested multigrid method (arXiv 2412.10910).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library never
calls it and shares no code with it: the oracle has its own basis functions,
quadrature, DoF numbering, assembly, point location and solver, written as the
slow, obviously correct definitions (assembled CSR matrices, an explicit
transfer matrix P built by brute-force point location, a textbook V-cycle).

Modules
  fe         1D Gauss-Lobatto Lagrange basis, Gauss-Legendre rules, Q1 map (Sec. 3.2, Sec. 4)
  dofs       continuous Q_k DoF numbering, Dirichlet set, support points (Sec. 2)
  assembly   element matrices and load vectors, Poisson and elasticity (Eq. problem, Sec. 4.4)
  transfer   point location + Newton inversion and the transfer matrix P (Eqs. pointwise..residual2, Sec. 3.1)
  multigrid  Jacobi diagonal, Lanczos, Chebyshev, Algorithm 1 V-cycle, Cholesky coarse solve, PCG (Sec. 4)
  hierarchy  glue: a whole level hierarchy with full-length vector helpers

Parity pins live in tests/test_oracle_*.py.  One function is "parity unpinned":
the CG iteration count under this project's solver settings (no number in the
paper applies; the paper uses an AMG coarse solver and a 1e-4 reduction).
"""
