"""FP64 CPU oracle of the additive overlapping DDM for the Helmholtz equation
(Leng & Ju, "An Additive Overlapping Domain Decomposition Method for the
Helmholtz Equation", 2018).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check of
the package entry file and the CPU-baseline leg of the benchmark may import it.
The product path (the CUDA library and its Python binding) never calls it and
shares no code with it: the two meet only through the seeded input arrays
drawn by ``paper_1807_04180_gb300.workloads``, which hold none of the method's
arithmetic.

Modules
-------
pml_operator  PML stretching (Section 2.1, Eq. (11)) and the J-scaled
              5-/7-point finite-difference PML operator (Eq. (9), Section 4).
ddm           Structured overlapping partition, cut-off and characteristic
              functions, transfer operators Psi (Section 2.2), Algorithm 3.1
              run as an iteration, the assembled DDM solution (Eq. (39)) and
              the global truncated problem solved directly (Section 3.1).
krylov        Right-preconditioned flexible GMRES with the DDM preconditioner
              (Section 4.2.2).

Every function works in complex128 / float64.  Pins that tie these functions
to the paper and to mathematics independent of them live in tests/
(test_oracle_*.py).
"""
