"""Plain, slow, FP64 CPU oracle for DoGIP on simplices (arXiv 1710.09913).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from here.  The
product path (the CUDA library and its Python binding) never imports, calls or
links this package, and this package imports nothing from the product path except
the seeded input generators (``paper_1710_09913_gb300.inputs``), which hold none of
the method's arithmetic.

Modules (each function cites the paper passage it follows):
  refelem     -- P_q Lagrange nodes and bases on the reference simplex (Section 2.1),
                 DoGIP interpolation tables B^ (Theorems 4 and 8), W-basis integrals
  topology    -- dof map l_T, Dirichlet boundary set, greedy element colouring
  quadrature  -- collapsed Gauss--Jacobi rules (Golub--Welsch) on the simplex
  assembly    -- conventional assembled sparse matrices (eqs. linsys_gp, linsys_se)
  dogip       -- A_T^DoGIP (Theorems 4 and 8), Algorithm 1, Jacobi diagonal
  solvers     -- Jacobi-PCG and FP64 iterative refinement with an FP32 inner solve
  gradient    -- compliance gradient with respect to element coefficients
  counts      -- memory / multiplication counts of Section 3 (eqs. memory_eff, comp_eff)

Parity status of each function is stated in its module docstring; everything is
pinned by the tests in ``tests/test_oracle_*.py`` except the FP32 emulation in
``solvers.iterative_refinement`` (parity unpinned: the paper fixes no precision).
"""
