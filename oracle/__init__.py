"""FP64 CPU oracle for the LM linear solve of "Multigrid for Bundle Adjustment".

Test infrastructure only.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import anything from here; the GPU library
never does, and this package shares no code with it (the seeded scene
generator is the one module both consume, and it holds none of the solver's
arithmetic).

Everything is plain NumPy/SciPy in float64, written to be checked against the
paper by eye:

* ``camera``    residuals and analytic Jacobians of the 9-parameter camera
                (the model the paper names in Section 6, in the convention of
                the BAL datasets it cites in Section 4).
* ``schur``     the damped normal equations of Section 2.1 (Eqs. 2-4), the
                explicit Schur complement ``S = A - F^T E C^-1 E^T F``, the
                implicit product of Section 3.6, reduced right-hand side and
                point back-substitution.
* ``multigrid`` Section 3: near-nullspace (3.1), visibility strength of
                connection and Algorithm 2 aggregation (3.2), tentative
                prolongator by per-aggregate QR (3.3), Galerkin coarse
                operators (Section 2.3), Lanczos eigenvalue estimate and
                Chebyshev smoother (3.4), and the V-cycle of Algorithm 1.
* ``pcg``       preconditioned conjugate gradients (Section 2.1/3.6).
* ``lm``        one Levenberg-Marquardt step (Section 2.1, Section 5 settings).
* ``adjoint``   gradient of the LM step through the linear solve.
* ``rng``       SplitMix64, the counter-based generator for the Lanczos start
                vector (Steele, Lea & Flood 2014).

Parity pins (what fixes each function independently of this code) live in
``tests/test_oracle_*.py``.
"""
