"""FP64 CPU oracle for the inverse-DFT hot path.  TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct reference that the CUDA
library is checked against.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import it; the library never calls it and
shares no code with it (the two have separate implementations of every step,
including the Gauss-Lobatto rules, the element matrices and the mesh
numbering).

Modules and the passages of the paper they follow:
  fe          spectral finite elements on a uniform box: GLL nodes (Sec. 3.2.1),
              Lagrange basis (Eq. 12), element matrices and assembly (Eq. 17),
              lumped mass and standard form H~ = M^-1/2 H M^-1/2 (Eq. 19).
  potentials  Hartree potential by an FE Poisson solve, LDA exchange (inputs).
  ks          lowest eigenpairs of H~ (Eq. 15/19), Fermi-Dirac occupations and
              chemical potential (Eq. 4, Eq. 5), density (Eq. 4).
  adjoint     loss (Eq. 1), adjoint right-hand side (Eq. 7, 10, 18, 20),
              MINRES on the complement of the null space (Sec. 3.2.2),
              component along psi (Eq. 8, 9), gradient (Eq. 11, 22),
              far-field mask (Sec. 3.1.2).
  lbfgs       limited-memory BFGS update of v_xc (Eq. 21).
  chebyshev   scalar Chebyshev recurrences used by the filter (Sec. 3.2.2).
  scf         self-consistent generation of a target density (input recipe).
  graded      graded tensor-product meshes (Sec. 4.2.2 reading): per-axis cell
              breaks refined towards the nuclei, per-cell scalars on the three
              Kronecker terms of K_e (Eq. 17), element orders up to 6.
  potential_matrix  dense per-cell potential matrices: the Gauss-quadrature
              reading of the potential term of Eq. 17 (the default collocates it).
  transfer    linear (Q1) v_xc mesh, transfer of v_xc to the orbital nodes and of
              the gradient back (Sec. 3.1.1, Sec. 3.2.2, Eq. 22).
  initial_guess  initial v_xc of Eq. 25 and Eq. 26: Slater or LB94 exchange plus
              PW92 correlation, blended with the scaled Fermi-Amaldi potential
              (Sec. 4.2.3); nodal density gradients of the FE interpolant.

Parity status of each function is stated in its docstring; every function has
at least one pin in tests/test_oracle_*.py (closed forms, brute force,
finite differences or library cross-checks).
"""
