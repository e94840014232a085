"""CPU FP64 oracle for the stochastic multiscale flux basis method.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
link this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code with the CUDA path; both read their inputs from ``sfb_workloads``.

The oracle is written from the paper (Ambartsumyan, Khattatov, Wang, Yotov,
"Stochastic multiscale flux basis for Stokes-Darcy flows", arXiv 1802.06263)
as plain, slow, obviously correct numpy/scipy code in float64:

* ``kl``          multi-region KL expansion of the log permeability
                  (Section 2.1, Eqs. 2.11-2.13, covariance Eq. 6.1);
* ``collocation`` Gauss-Hermite rules, tensor and Smolyak grids, the global
                  to local index map (Section 4, Section 5.4 Step 4);
* ``mortar``      mortar spaces and the L2 projections onto subdomain traces
                  (Section 3.3, Section 5.2 action of S_H);
* ``darcy``       lowest-order RT on rectangles with trapezoidal quadrature,
                  i.e. cell-centred finite differences, and its
                  Dirichlet-to-Neumann map (Eqs. 5.5-5.8);
* ``stokes``      Taylor-Hood P2-P1 with the BJS condition and normal-stress
                  mortar data (Eqs. 2.10, 5.1-5.4);
* ``coupled``     the monolithic mortar system (Eqs. 4.2-4.4), the interface
                  problem (Eqs. 5.9-5.10), Methods S1, S2, S3 (Section 5) and
                  the statistical moments (Eq. 2.1).

Every function carries a pin in ``tests/test_oracle_*.py`` against closed
forms, invariants, brute force or values the paper prints. Functions without
such a pin say "parity unpinned" in their docstring.
"""
