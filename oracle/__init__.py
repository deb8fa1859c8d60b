"""Plain FP64 CPU oracle of the FR hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything here; the product path (the CUDA library and
its Python binding) never does, and shares no code with it.

Modules: ``basis`` (Gauss-Legendre points, Lagrange, DG correction),
``element`` (tensor reference element and dense operators), ``geometry``
(element maps, metrics, face connectivity), ``physics`` (Navier-Stokes
fluxes, Rusanov and Roe interface fluxes, boundary states), ``fr`` (residual,
BR2 or LDG viscous terms), ``fr_var`` (residual with a degree per element,
mortar coupling of unequal faces), ``timestep`` (RK4, LSRK45, the
Bogacki-Shampine 3(2) pair with its error-per-step controller),
``acoustics`` (probe, OASPL).
"""
