"""FP64 CPU oracle for the eddy-current A-V finite-element method.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the method computes, written from the paper's equations
(Sec. 2-3) and the readings stated in each module's notes (where the paper
is silent, garbled or ambiguous).  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA library and never imports it; the two
meet only in the seeded input generator ``ect_inputs``.

Modules
  fem        element matrices (Eq. sesquil / L11-L22), scalar CSR assembly,
             A.n = 0 elimination, V identity rows, symmetric scaling
  rhs        coil source term J (Sec. 4) and its mass-matrix load
  solve      dense LU, SuperLU, block-Jacobi inverse, (F)GMRES with CGS2
  impedance  Delta Z by reciprocity and by coil EMF (Eq. impedkl, impedmod)
  mlp        FP64 reference MLP for the surrogate (forward, backward, Adam)

Pins: every function is pinned by closed forms, invariants, special cases
that reduce to a textbook routine and brute force on tiny inputs (see tests/,
the test_oracle_* files).  The paper prints no field or impedance value, so
no pin is a number copied from it.
"""
