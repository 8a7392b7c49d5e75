"""FP64 CPU oracle for the locally relaxed entropy-stable RK step.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (the CUDA library and its Python binding) never imports,
links or executes anything here, and this package never imports the product.

It is a plain, slow, obviously correct restatement of the method of Ranocha,
Dalcin and Parsani, "Fully-discrete explicit locally entropy-stable schemes
for the compressible Euler and Navier--Stokes equations" (2020):

* ``sbp``    -- LGL nodes/weights and the diagonal-norm SBP derivative
                (Section 3.1, text around Eq. (compressible_ns_diss)).
* ``gas``    -- ideal-gas thermodynamics, entropy S = -rho s, entropy
                variables w = dS/dq (Section 3.1), the Ismail--Roe
                entropy-conservative two-point flux with the series
                logarithmic mean, Rusanov interface dissipation, the
                Navier--Stokes viscous flux.
* ``dg``     -- the semidiscretisation of Eq. (compressible_ns_diss) on a
                periodic Cartesian hexahedral mesh: volume flux differencing,
                interface SATs, BR1 viscous terms; local entropies
                eta_kappa = 1^T P S_kappa (Section 3.2).
* ``rk``     -- explicit RK step, Eq. (RK-step), with the entropy estimate of
                Eq. (eta-est-1-RK); Butcher tableaux BS3 and RK4 (Section 4).
* ``relax``  -- the per-element relaxation equation, the last row of
                Eq. (relaxation-local-gamma), its root gamma_kappa, and
                gamma = min_kappa gamma_kappa (Theorem 2.3).

Every array is float64.  Where the paper is silent the module docstrings state
the reading taken.
"""
