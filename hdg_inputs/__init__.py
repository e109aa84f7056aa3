"""Seeded synthetic inputs for the HDG trace solver.

This package produces the *inputs* of the solver's hot path: meshes with their
face connectivity, and the per-element HDG blocks A..J, r_u, r_uhat of the
linearised system (Welter & Nguyen, Sec. 2.3, Eq. matrixform; Sec. 4.1, Eq.
w16 for the q-equation blocks M, B_d, C_d).  Both the CUDA library and the
FP64 oracle consume these arrays; neither static condensation, assembly, the
preconditioners nor GMRES live here.

Modules:
  basis     -- 1D/2D/3D Lagrange bases and Gauss quadrature
  mesh      -- structured triangle and (perturbed) hexahedral meshes, faces
  blocks    -- element blocks for Poisson, linear elasticity and a
               convection-diffusion-reaction system
  workloads -- the five named workloads with their seeds
"""
