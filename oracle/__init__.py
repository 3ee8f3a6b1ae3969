"""CPU FP64 oracle for the spectral-element tropical-cyclone hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark use it.  It is a plain, slow, obviously
correct restatement of the discretisation of arXiv 2410.21607 (Tissaoui,
Guimond, Giraldo, Marras, "Accelerating Simulations of Tropical Cyclones using
Adaptive Mesh Refinement"):

  basis.py      LGL points/weights, Lagrange basis, derivative, 2:1
                interpolation and exact mass matrices (Sec. 3)
  mesh.py       brute-force mesh, global nodes and the hanging-node
                constraint matrix Q (Sec. 3.1, "modified DSS")
  refstate.py   hydrostatic reference state (Eqs. rho_split..hydro_bal)
  rhs.py        right-hand side of the split Euler equations, conservative
                and non-conservative sets (Eqs. mass_split..ent_split, Sec. 3)
  rk.py         explicit third-order Runge-Kutta (Sec. 4, time integration)
  adapt.py      threshold criterion and the refine/coarsen/balance update
                (Sec. 3.1-3.2, Algorithm 3)
  transfer.py   solution transfer on refinement/coarsening
  diag.py       maximum-wind diagnostics (Sec. 4.2)

Every array here is numpy float64.  The oracle shares no code with the CUDA
library and never imports it.
"""
