"""CPU oracle for the parallel CLS hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 restatements of what the paper defines, used to check the
CUDA path.  Only the tests, the package smoke check and the benchmark's CPU
baseline leg may import this package; the product path never calls it.  It
shares no code with the CUDA library (only the seeded generators in
`workloads` serve both sides).

Modules
  spectra   truth tables sp_t of the symmetric constraint types (Sec. 2.1
            Eq. 3's sp_i; Sec. 2.2 / Table 2 PB forms)
  fe        Walsh-Fourier expansion FE and its gradient: brute-force
            definition (Eq. 1) and the FP64 Poisson-binomial DP
  exact     exact-rational coefficients: Eq. 3 and the Appendix A closed
            forms; elementary-symmetric-polynomial evaluation (Eq. 2)
  cls       whole-problem objective/gradient (Sec. 2.3, Eq. 5), projected
            step, rounding and exact satisfaction count, Philox init

Parity status: every function here is pinned by tests/test_oracle_pins.py
against an independent route (brute force over corners, exact rationals,
closed forms, identities, a library generator) except where a function's
docstring says "parity unpinned".
"""
