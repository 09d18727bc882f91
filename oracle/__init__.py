"""FP64 CPU oracle for the stochastic Galerkin KKT solve (test infrastructure).

This package is test infrastructure.  Only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the library's product path never
does, and it shares no code with the CUDA path.  Every function is a plain,
slow restatement of the paper (Li, Onwunta, Sousedik, "Stochastic Galerkin
Method and Hierarchical Preconditioning for PDE-constrained Optimization") in
float64 with NumPy/SciPy, citing the section/equation/algorithm it follows.

Modules
  basis     graded multi-index set, Legendre triple products G_k      (Sec. 2)
  fe        Q1 stiffness K_k and mass M on the unit square            (Sec. 2, Eq. (gPC-A))
  operators SG operator sum_k G_k (x) K_k, KKT systems, right-hand sides (Eqs. (stoch-system), (KKT:stoch-time-dependent))
  precond   Chebyshev mass solve, V-cycle, hGS sweep, block preconditioners (Eqs. (stoch-prec), (precon for time), Alg. 1)
  krylov    preconditioned MINRES and flexible GMRES with the stopping rule used by the library
  solve     end-to-end solves and dense direct reference solutions

Parity status: every function is pinned by tests in tests/test_oracle_*.py
except the Krylov iteration counts themselves, which are pinned only against
scipy's MINRES / GMRES, the minimal-residual property of GMRES and the
3-iteration ideal-preconditioner case.
"""
