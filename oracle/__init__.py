"""Oracle: a plain, slow, CPU restatement of the RS-CGC preconditioned FGMRES
solver for the Helmholtz equation, in complex FP64 (NumPy / SciPy).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package; only the test suite, the smoke entry point and the
benchmark's CPU-baseline leg use it.  It shares no code with the CUDA path: the
two meet only in the seeded inputs of ``workloads``.

Every function cites the passage of the paper it follows (Yovel & Treister,
"Scalable Multigrid Solver for the Helmholtz Equation: Real-Shifted Coarse Grid
Correction").  Where the paper is silent the reading taken is stated in the
docstring.

Modules
-------
grid        node grids, absorbing-layer profile, coefficient field   (Sec. 1, Sec. 5)
operators   fine operators: 2nd-order 5/7-point, compact 4th-order 9/19-point (Sec. 3.1)
transfers   full-weighting / bilinear and cubic grid transfers           (Eq. intergrid, levdep)
hierarchy   Galerkin coarsening and the real-shifted coarsest operator    (Eqs. Galerkin, realShift, CoarseRealShifted)
smoothers   damped Jacobi and red-black point relaxation                  (Sec. 2)
cycle       3-level V/W cycle, exact coarsest solve                       (Algorithm TwoGrid, Sec. 2)
krylov      flexible GMRES with right preconditioning                     (Sec. 5)
adjoint     least-squares misfit and its gradient w.r.t. slowness squared
dispersion  grid-to-grid dispersion analysis and the optimal real shift   (Sec. 4)

Parity status: every module is pinned by ``tests/test_oracle_*.py`` against
closed forms, brute-force dense constructions or the paper's printed tables,
except where a docstring says "parity unpinned".
"""
