"""Plain CPU oracle for the P-ERRK multirate stage loop (test infrastructure).

This package is test infrastructure only.  It is imported by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` and by nothing else; the product library never calls it and has
no fallback to it.  It shares no code with the CUDA path: the only common
module is ``workloads`` (seeded meshes and initial states, no method
arithmetic).

Everything is float64 numpy written from the paper (arXiv 2507.04991,
"Paired Explicit Relaxation Runge-Kutta Methods") and the textbook DGSEM it
cites:

* ``lgl``      Legendre-Gauss-Lobatto nodes, weights, differentiation matrix.
* ``physics``  Burgers / Euler fluxes, two-point EC fluxes, Rusanov dissipation,
               the paper's entropy s = -rho log(p rho^-gamma) (eq.
               EntropyMathematical) and its entropy variables (eq.
               EntropyVariables); the Navier-Stokes-Fourier viscous flux
               from entropy-variable gradients (Sec. 4.3.2).
* ``dgsem``    metric terms, the flux-differencing DGSEM right-hand side and
               the BR1 gradient and divergence of the viscous terms.
* ``tableau``  P-ERK Butcher archetypes (eq. PERK_ButcherTableauClassic_p2_E36,
               eq. PERK_ButcherTableauOwn_p3, eq. PERK_ButcherTableau_p4),
               order conditions over coloured rooted trees, stability
               polynomial, members built from a given stability polynomial
               (Sec. 2.2).
* ``perrk``    the partitioned RK stage loop in full Butcher form (eq.
               PartitionedRKSystem), Delta H (eq. EntropyChange_EntropyVariables_ReArranged),
               the relaxation equation and its Newton, bisection and secant
               solves (eq. RelaxationEquation, Sec. 3.1) and the relaxed
               update (eq. RRKM_Update).
* ``mlp``      2x64 tanh MLP forward / backward / Adam for the learned gamma guess.

Pins (what each part is checked against, in ``tests/test_oracle_*.py``):
closed-form LGL data, SBP property, polynomial exactness, complex-step
derivatives of the entropy, Tadmor's entropy-conservation condition,
conservation / entropy conservation / free-stream preservation of the RHS,
brute-force order conditions, textbook special cases (midpoint, SSPRK3), the
closed-form gamma for a quadratic entropy, observed convergence order and
finite-difference gradients; for the viscous part the paper's traveling
viscous shock as an exact discrete solution, frame indifference, Stokes'
hypothesis and the BR1 entropy identity; for polynomial-built members the
stability polynomial of the full Butcher matrix.  No function here is
"parity unpinned".
"""
