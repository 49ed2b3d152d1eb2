"""CPU FP64 oracle for the space-time multigrid method of Gander & Neumueller
(arXiv:1411.0519), "Analysis of a new space-time parallel multigrid algorithm
for parabolic problems".

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may use it.  It shares no code, tables or constants with the CUDA path: every
matrix here is assembled from its integral definition by Gauss quadrature and
every solve is a plain sparse direct solve (SciPy SuperLU) or a dense NumPy
solve.  It is deliberately slow and written so that each step can be compared
with the paper by eye.

Modules
  dg_time    -- DG-in-time element matrices K_tau, M_tau, N_tau (Section 1)
  fe_space   -- P1 / Q1 mass and stiffness matrices M_h, K_h (Section 1)
  spacetime  -- block system L u = f, load vector, initial-condition term
                (Section 1, system (chap4_generalLinearSystem))
  transfer   -- restriction / prolongation in time and space
                (Section 3.2, eqs. (chap4_restrictionTime),
                (chap4_spaceRestrictionProlongation))
  hierarchy  -- Pade stability function, critical parameter mu*, coarsening
                rule (Remark chap4_remarkCriticalDiscretizationParameter,
                Section 4)
  multigrid  -- damped block-Jacobi smoother, V-cycle, solve, forward
                substitution, adjoint (Section 2, eq. (chap4_smoother))
  lfa        -- local Fourier mode analysis: symbols of L, S, R, P and the
                two-grid iteration matrices (Section 3, Lemmas 17-29,
                Theorems 5-6)
  simplex    -- P1 on the paper's simplicial meshes (unit square in 4
                triangles, unit cube in 12 tetrahedra, refined uniformly;
                Section 4, Examples 1 and 2): assembly by quadrature and the
                nested-space prolongation
  mesh_multigrid -- the space-time hierarchy, coarsening rule and inexact
                block inverse on those meshes (the cycle of ``multigrid``)

Parity status: every function above is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except the numerical values of the LFA two-grid
curves themselves, whose figure data are missing from the paper ("parity
unpinned" for the curve values; the bounds the paper states are pinned).
"""
