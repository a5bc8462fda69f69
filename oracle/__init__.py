"""Plain CPU FP64 oracle of the agglomeration-based multigrid PCG solver for
the SIPG-DG monodomain model (arXiv 2602.16312).

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import or run it.
The product path (the CUDA library and its binding) never imports it, and it
shares no code with that path: only the seeded input generators in
`paper_2602_16312_gb300.workloads` serve both.

The oracle is written for a reader checking it against the paper:
numpy/scipy in float64, library primitives (sparse products, dense
factorisations, eigen-solvers) used as steps, no blocking or fusion.

Modules
  refelem    reference element: GLL nodes, Lagrange basis, Gauss rule (Sec. 3)
  sipg       SIPG stiffness A, mass M and A0 = c M + A (Sec. 3, Eq. fully_discrete)
  multigrid  agglomerated levels, prolongation, Galerkin coarse operators
             (Eq. inherited_matrices, Algorithm 3), block-Jacobi Chebyshev
             smoother, V-cycle, PCG (Sec. 5-6)
  monodomain ionic models (Sec. 2.3), IMEX time step (Sec. 3.1), adjoint

Parity status per function is stated in each module header. Functions that
follow a reading of the paper (not a closed form) say so.
"""
