"""Plain FP64 CPU oracle for the LDG Stokes multigrid V-cycle (test infrastructure).

This package is the slow, obviously-correct reference that the CUDA library is
checked against.  It is test infrastructure only: nothing in the product path
(the C-ABI library and its Python binding) imports, links or runs it.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark use it.

It shares no code with the CUDA path.  Its inputs (problem data, seeded random
vectors) come from ``paper_1911_05888_gb300.problems``, which holds no part of
the method.

Modules:
  basis      Legendre basis, Gauss quadrature, 1-D element matrices.
  ldg        Appendix A: fine-mesh LDG operators (M, M_mu, M_rho, G_k, E~, E) and RHS.
  hierarchy  Appendix B: operator coarsening (Algorithms 2 and 3) and the
             Stokes block operator of eq. (blockform) / (timedep2) per level.
  multigrid  Section 3: block Gauss-Seidel (multi-coloured and lexicographic),
             Algorithm 1 V-cycle, bottom solver, outer iteration, GMRES and the
             convergence rate of eq. (rho); mixed-precision emulation.

Every function states the passage of the paper it follows.  Where the paper is
silent the reading taken is stated in the docstring.
"""
