"""CPU oracle for the Wilson-fermion PF/Hasenbusch HMC hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 (optionally
extended-precision) restatement of what the method computes, written from
the paper (Haar, Kamleh, Zanotti, Nakamura, "Improving polynomial-filtered
Hybrid Monte Carlo with Hasenbusch", INPC 2016): Section 2 (lattice action,
HMC steps, two-flavour fermion action and force, mass preconditioning,
polynomial filtering), Section 3 (cost metric, leapfrog, nested and
generalised multi-scale integration), Section 4 (PF-MP and three-filter
actions).  It shares no code with the CUDA path; only tests/, the smoke
check and bench.py's CPU-baseline leg may import it.

Modules
  lattice   geometry, shifts with the antiperiodic time boundary, parity
  dirac     gamma matrices (DeGrand-Rossi chiral basis)
  su3       generators, exponential (Taylor, scaling and squaring), projections
  wilson    D, D^dag, M, M^dag, even-odd M_hat, K_hat
  cg        conjugate gradient
  poly      Chebyshev filter polynomial (roots, normalisation, application)
  actions   pseudofermion actions and heat bath per action term
  force     fermion force and gauge force
  hmc       T/S steps, leapfrog, Omelyan 2MN, nested and generalised schemes,
            Hamiltonian, Metropolis
  philox    counter-based Gaussian draws (Philox4x64-10)

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, dense linear algebra on 2^4 lattices, finite
differences in extended precision or library routines, except where a
module docstring says "parity unpinned".
"""
