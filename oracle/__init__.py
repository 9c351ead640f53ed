"""Plain, slow FP64 CPU oracle of the adaptive multigrid solver.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package; the product path
(the CUDA library and its Python binding) never does, and this package never
imports the product path.  The two share no code; only the seeded input
generators in ``workloads`` serve both.

Contents, each following the paper (Brannick, Brower, Clark, Osborn, Rebbi,
"Adaptive Multigrid Algorithm for the QCD Dirac-Wilson Operator", 2007):

* ``wilson``    -- the Wilson-Dirac operator D of Sec. 1 (display after
                   Eq. 1), its adjoint, the normal operator A = D^dagger D,
                   and explicit sparse/dense matrices of D for small lattices.
* ``multigrid`` -- geometric blocking S_j (Sec. 3), chirality-split block
                   orthonormalisation of the relaxed vectors (Sec. 3, Eq. P1),
                   prolongation P and restriction P^dagger (Sec. 2), the
                   Galerkin coarse operator P^dagger A P (Eq. Galerkin), the
                   frozen two-step minimum-residual smoother (Sec. 4), the
                   five-step V-cycle (Sec. 2), the exact coarsest solve, and
                   the adaptive setup relaxation (Eq. relax) and the adaptive
                   refinement by V-cycles (Sec. 3).
* ``krylov``    -- plain CG and MG-preconditioned CG (Sec. 4).
* ``critical``  -- the critical-mass finder used to choose near-critical
                   masses (Sec. 4, mass gap m - m_crit).
* ``smoothed``  -- smoothed aggregation: the Richardson step on the vectors
                   before the prolongator is formed, its damping minimising
                   the condition number of the coarse operator (Sec. 3).

Every function states the passage it follows.  Pins against the paper and
the mathematics live in ``tests/test_oracle_*.py``; parity of any function
not pinned there is stated as "parity unpinned" in its docstring.
"""
