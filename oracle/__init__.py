"""Plain, slow FP64 CPU oracle of the EBIT phase-change time step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may call it.  It shares no code with the CUDA path (the only
common module is the seeded input generator ``paper_2402_13677_gb300.workloads``,
which holds none of the method's arithmetic).

Each module restates one part of the paper (arXiv 2402.13677) in the paper's
order and notation:

  geometry.py  Color-Vertex reconstruction (Sec. 2.1), volume fractions
               (property-average equation), narrow band (Sec. 2.4), ghost-fluid
               link fractions theta (ghost-temperature equation).
  sweep.py     interfacial velocity at markers (interfacial-velocity jump
               equation + bilinear interpolation, Fig. 2) and the dimension-split
               EBIT marker advection (marker-motion equations, Fig. 1).
  energy.py    WENO3 energy advection, narrow-band extension (extrapolation
               equation), the sharp T = T_sat implicit diffusion solve
               (ghost-temperature / Txx equations) and the interface heat and
               mass flux (mass-flux and normal-gradient equations).
  flow.py      ghost velocities (ghost-velocity equation), momentum predictor
               and projection (discretization equations 1-5, ghost-fluid Poisson
               equation).
  step.py      state, the five-step time iteration of Sec. 2.5 and the
               diagnostics of Sec. 3 (M_d, M_c, vapour volume).

Every linear system is assembled explicitly and solved with a sparse direct
solver (scipy.sparse.linalg.spsolve), so the oracle carries no iteration error.
"""
