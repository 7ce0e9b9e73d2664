"""FP64 CPU oracle for the hyper-power preconditioned Stokes solve (arXiv 2311.06926).

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously-correct restatement of what
the paper's method computes, used only by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``. The product (the CUDA library and
its Python binding under ``paper_2311_06926_gb300/``) never imports it, and this package never
imports the product: the two share no code, tables or constants.

Modules
  basis      open knot vectors, Cox-de Boor B-splines, unit-integral M-splines (App. B.1)
  univariate the 1D matrices M, K, C, M-check, K-check, C-check, N-check, B-check, T-check
             (App. B.3 and Sec. 3.3)
  stokes     assembled Kronecker blocks A, B and the saddle matrix (Sec. 3.3, Eq. 3.3),
             the Nitsche lid load and body-force load, pressure normalisation
  quadrature brute-force 3D Gauss quadrature of the weak form (Sec. 3.1-3.2), an independent
             route used only to pin the Kronecker assembly
  precond    fast diagonalisation P_V0^-1 (App. A.4, Sec. 4), pressure mass P_Q0^-1 (Sec. 4),
             the hyper-power recursion for the V and Q blocks (Eqs. 2.1, 4.4-4.6)
  krylov     preconditioned MINRES (the benchmark solver of Sec. 5) and flexible GMRES
  matfree    matrix-free mode-product variants of A, B used at meshes too large to assemble

Every floating-point quantity is float64.
"""
