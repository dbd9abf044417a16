"""CPU FP64 oracle for the matrix-free GMG Stokes hot path (arXiv 1907.06696).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call, link
or execute this package: only the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline / reference arm use it. It shares no code with the
CUDA library; the only common module is `sinker_inputs` (seeded inputs, no
method arithmetic).

Everything here is written from the plain definitions in the paper, in FP64,
with no blocking, fusion or reordering beyond what the definitions state:

* fe.py        Q2/Q1 bases, 3-point Gauss quadrature and element matrices by
               full quadrature (Section 2.1, weak form and block definitions).
* mesh.py      uniform n^3 hexahedral mesh, DoF numbering, Dirichlet sets.
* sinker.py    sinker viscosity and forcing (Section 3.2) and the viscosity
               averaging / level restriction (Section 2.3).
* operators.py element-by-element and CSR application of A, B, B^T, M_p, the
               right-hand side F and the diagonal of A.
* gmg.py       level hierarchy, Q2 prolongation/restriction, Jacobi-Chebyshev
               smoothing, Lanczos eigenvalue estimate, V-cycle (Section 2.2.1).
* krylov.py    Schur approximation (Section 2.2.2), block-triangular
               preconditioner (eq. stokes_precond), FGMRES(50) and dense solves.
* octree.py    adaptive octree: refinement in shells around the sinkers, 2:1
               balance, hanging-node constraints, level structure of local
               smoothing (refinement-edge nodes, copy levels).
* adaptive.py  active operators with constraints (C^T E C), right-hand side,
               level operators and transfers, local-smoothing V-cycle.

Parity pins live in tests/test_oracle_*.py. Functions with no independent pin
say "parity unpinned" in their docstring.
"""
