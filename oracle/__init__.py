"""Plain float64 CPU oracle of the bundle-adjustment normal-equation solve.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
the benchmark's CPU-baseline leg may import it.  The CUDA library never calls
it, and it shares no code with the library: only the seeded scene generator
(``paper_2110_04015_gb300.synthetic``, which holds none of the method's
arithmetic) feeds both.

It is a slow, direct statement of what the paper computes, in the paper's
order and notation (Weber, Demmel, Cremers, "Multidirectional Conjugate
Gradients for Scalable Bundle Adjustment", GCPR 2021):

* ``camera``  - the BAL reprojection residual r_i(x) and its Jacobian blocks
  J_p, J_l (Section 3.1, Eqs. 1-4; the camera formula is the BAL model's,
  which the paper uses but does not print).
* ``normal``  - the damped normal equation H, U_lambda, V_lambda, W, b_p,
  b_l (Eqs. 5-11).
* ``schur``   - the reduced camera system S, b~ (Eqs. 12-14) and the dense
  brute-force elimination used to pin it.
* ``solvers`` - block-Jacobi PCG (Algorithm 1) and MCG (Algorithm 2) with the
  tau-test, the pseudo-inverse, full reorthogonalisation and the Q update of
  Eq. 18.
* ``lm``      - back-substitution (Eq. 15, sign corrected) and one
  Levenberg-Marquardt step (Section 4.1).

Every function is pinned by ``tests/test_oracle_*.py`` against something
other than itself: finite differences, dense textbook eliminations and
solves, closed forms and invariants.  Parity status per function is listed in
each module's header.
"""
