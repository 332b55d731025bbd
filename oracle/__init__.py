"""Plain, slow, obviously-correct FP64 CPU oracle for the LFRic pressure/mixed solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` use it.  It shares no code with the CUDA library (``csrc/``): the only
common module is ``synthetic`` (seeded random inputs, no solver arithmetic).

Modules (each function cites the passage of Maynard, Melvin & Mueller, "Multigrid
preconditioners for the mixed finite element dynamical core of the LFRic atmospheric
model", arXiv 2002.00756, that it follows):

  geometry   equiangular cubed-sphere column mesh (Sec. 5.1 mesh; shallow atmosphere)
  helmholtz  Helmholtz operator H (Eq. helmholtz_operator, strong volume-normalised
             form), its column tridiagonal part H_z-hat and the block-Jacobi sweep
             (Eq. jacobi) with the textbook Thomas algorithm
  multigrid  horizontal-only hierarchy, prolongation (Eq. prolongation), restriction
             (its dual), rediscretised coarse operators and the V-cycle (Algorithm 1)
  krylov     restarted, right-preconditioned GCR (Sec. 4.1, Sec. 5.1)
  mixed      reduced (u, p) mixed operator and the approximate Schur-complement
             preconditioner (Sec. 3.4, Steps 1-3)
  reference  assembled sparse / dense matrices and direct solves (the plain definition
             of the solution of the linear systems)

Parity status: the V-cycle contraction factor and the mixed-solve iteration counts are
"parity unpinned" (the paper prints neither for this synthetic operator); every other
function is pinned by tests/test_oracle_*.py against closed forms, invariants, library
special cases or dense direct solves.
"""
