"""Plain FP64 CPU oracle for the tree-based dGSEM hot path (test infrastructure only).

This package is the checker, not the product.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It shares
no code with the CUDA library in ``paper_2404_16648_gb300`` and never imports it.

Modules (each function cites the passage of arXiv 2404.16648 it restates):

* ``basis``   -- LGL nodes/weights, collocation derivative, L2 projection matrices
                 (Sec. 3.3: solution transfer and fluxes on non-conforming faces).
* ``physics`` -- Euler fluxes, equation of state, hydrostatic background, Rusanov flux
                 (Sec. 2.1 Eq. 1 / Eq. "eulervector", Sec. 2.2, Sec. 4.3).
* ``forest``  -- forest of quad/oct-trees with active-leaf storage, regrid with buffer B,
                 2:1 balance, conforming/mortar/boundary face lists (Sec. 3.1, 3.2.1, 4.3).
* ``dg``      -- strong-form dGSEM right-hand side with mortars, SSP-RK3, conservative
                 parent<->child transfer, integrals, initial conditions (Sec. 2.2, 3.3, 4.3),
                 and the BR1 reading of the artificial viscosity named in Sec. 4.3.
* ``adjoint`` -- the discrete adjoint of the right-hand side and of the SSP-RK3 step by
                 complex-step Jacobian columns, and the gradient of the final kinetic energy
                 with respect to the initial theta' field.

Parity status of each function is stated in its docstring; every function here is pinned by
``tests/test_oracle_*.py`` against closed forms, invariants or brute force, except the
end-to-end multi-step fields, for which no published values exist ("parity unpinned" beyond
the invariants listed in those tests).
"""
