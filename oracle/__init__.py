"""CPU reference (oracle) for the RT-CC3 triples hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call,
link or execute anything under ``oracle/``; only ``tests/``, the smoke check
in ``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.  It shares no code with the CUDA path: the only module
both sides import is the seeded input generator
``paper_2407_18947_gb300.synth``, which holds no arithmetic of the method.

Modules
-------
``cc3``         plain complex128 PyTorch-CPU restatement of RT-CC3 (the
                paper's Section 2 and Appendix A): T1 dressing, the CCSD part
                of the residuals, the triples (Eqs. 4, 6, A25 read per the
                commutator), X1/X2 (Eqs. A21, A22), the Lagrangian (Eq. A6)
                and its Euler-Lagrange derivatives (Eqs. A10-A15), density and
                dipole, RK4 and the ground-state solve.
``explicit``    the paper's printed lambda-side formulas (lambda_3 Eq. A26,
                Y1 Eq. A23, Y2 Eq. A24, triples density Eqs. A31-A33), with
                the readings of two garbled Y1 terms; compared with the
                Lagrangian derivatives of ``cc3`` to 1e-12
                (``tests/test_oracle_explicit.py``).
``bruteforce``  second quantisation in the full N-electron determinant
                space for tiny systems: the pin for every convention.
``finite_field`` the finite-difference stencils of Eqs. 19-20.

Parity status: every function is pinned by a test in ``tests/``:
``cc3`` against brute force (``bruteforce``), exact two-electron time
evolution, finite differences of the brute-force Lagrangian, stationarity and
Hellmann-Feynman; ``explicit`` and the lambda side of ``cc3`` against each
other (two independent routes); ``finite_field`` against exact polynomials.
None is "parity unpinned".
"""
