"""Oracle for the outer-region R-matrix hot path (R -> K -> Omega).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow CPU restatement of
what the GPU path computes, written from the paper (Section "Overview",
Eqs. radial, match, wnk, rmatrix; Section "Glossary of terms" for T and
Omega; Section "namelist stgf MQDT variables" for closed-channel
elimination). Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg may import it. It shares no code with the CUDA library and does
not import the product package.

Floating point is IEEE double throughout, except the special functions of
oracle/coulomb_ref.c, which are evaluated in binary128 and rounded to double.
Linear algebra uses numpy/LAPACK (LU with partial pivoting) as a library
primitive.

Parity status per function (what pins it, in tests/test_oracle_pins.py):
  coulomb functions     mpmath coulombf/coulombg, Wronskian, eta = 0 closed forms
  closed log-derivative mpmath whitw, hydrogenic integer-nu closed forms
  regular_analytic      Gamow-factor relation to F at positive energy, also
                        3e-7 Ry above threshold and inside an l = 15
                        barrier (tests/test_oracle_threshold.py)
  near-threshold        tests/test_oracle_threshold.py: s / sqrt(A), c sqrt(A)
  analyticity           continue into f and g at half-integer nu across the
                        threshold; theta ~ A f cos(pi nu) - g sin(pi nu)
  r_matrix              brute-force mpmath sum, exact symmetry, single-pole limit
  k_direct              one-channel hand formula, square well vs closed-form
                        tan(delta), 1 open + 1 closed closed form, symmetry,
                        unitarity of S
  k_mqdt                identity with k_direct (exact elimination identity)
  t_matrix / omega      optical theorem, symmetric Omega, real-form |T|^2
  qdt (coarse-mesh      tests/test_oracle_qdt.py: every energy a node equals the
  interpolation)        plain MQDT solve; a node matrix linear in energy is
                        reproduced exactly (also when extrapolating); error
                        of S_u interpolation falls as h^2; segment and
                        qetest rules on hand-made grids
  propagate (outer-     tests/test_oracle_propagate.py: without coupling K at r1
  region propagation    equals K at a; free s-wave closed form; dipole tail
  with multipoles)      A/r^2 against Bessel J, Y of order sqrt(A + 1/4) and
                        quadrupole tail A/r^3 at threshold against I_1, K_1
                        (planted mistakes in the power, the signs of U, eps
                        and b each fail one); round trip a -> r1 -> a; an
                        independent RK4 converges to it at fourth order;
                        sector lengths do not change K
  many-channel          tests/test_oracle_pins.py: interleaved channel groups
  structure             that share no poles give a block-diagonal K whose
                        blocks and collision strengths equal each group
                        solved alone (direct and MQDT); relabelling the
                        channels permutes K and the level pairs of Omega
  cross-threshold K, Omega beyond these checks: parity unpinned (the paper
                        prints no K or Omega values for any system).
"""
from .rmatrix import (  # noqa: F401
    RM_OK, RM_ETHRESHOLD, RM_ENEAR_POLE, RM_ESINGULAR, RM_ECF_NOCONV,
    MODE_DIRECT, MODE_MQDT,
    channel_functions, r_matrix, match_direct, mqdt_set, match_mqdt,
    t_matrix, omega_add, solve_energy, solve_energies, tri_index,
)
