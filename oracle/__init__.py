"""CPU FP64 oracle for MGRIT applied to method-of-lines linear advection
(De Sterck, Falgout, Krzysik, Schroder: "Efficient multigrid reduction-in-time
for method-of-lines discretizations of linear advection", arXiv 2209.06916).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or link this package; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py`` use it.
It shares no code, tables or constants with the CUDA path: every coefficient is
derived here again from the paper's definitions.

Modules
  coefficients  upwind taps (Sec. 4.1), e_FD (Eq. e_FD_def), RK stability
                functions and tableaux (Sec. 4.2), SL stencil and f_{p+1}
                (Sec. 3, Lemma 3.1), difference matrices D (Eq. Dp+1_def),
                correction constants phi (Lemma 6.1, Sec. 6.2 multilevel recursion).
  operators     Phi = R_q(-c L_p) (Eq. MOL_M_def) applied through RK stages,
                S_p (Sec. 3), Psi = (I - phi D)^{-1} S_p (Eq. MOL-SL-corrected).
  mgrit         sequential time-stepping (Eq. one-step-general), two-level and
                V-cycle linear MGRIT (Sec. 2.2) with F / FCF relaxation.
  gmres         GMRES from a zero guess with the Sec. 6.3 stop rule, for the
                approximate correction solves of the coarse operators.
  lfa           two-level LFA convergence factor (Eq. rho-asym).
  rng           SplitMix64 counter-based uniform generator for the random
                initial MGRIT iterate (Sec. 5.3 numerical setup).

Parity status per function is stated in each module's header; the pins live
in tests/test_oracle_*.py.
"""
