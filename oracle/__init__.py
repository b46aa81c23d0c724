"""FP64 CPU oracle for the FNPF-SEM hot path (arXiv 2506.09435).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of what the GPU path computes, written from the paper's
mathematical model (Sec. 2, Eqs. Laplace_strong, kinematic/dynamic free-surface
conditions), its weak forms (Sec. 3.1.1, Eqs. Laplace_weak, free_surface_weak),
the mesh construction (Sec. 3.1.2), ERK4 (Sec. 3.2), relaxation zones (Sec. 3.3)
and the workflow (Sec. 3.4, Steps 4.1-4.7).  Only the test-suite, the smoke
entry point and the benchmark's CPU-baseline leg may import it.  It shares no
code with the CUDA library and never imports it.

Modules
  gll      -- Gauss-Lobatto-Legendre rule and differentiation matrix
  mesh     -- extruded structured hexahedral (or 2D quad) mesh, node numbering
  operator -- stiffness operator by its quadrature definition, sparse assembly
  solve    -- Dirichlet-Neumann Laplace solve, vertical velocity recovery
  surface  -- Zakharov right-hand side, ERK4, relaxation, diagnostics
  tlm      -- exact tangent-linear model of one RK4 step (complex step)
  filter   -- modal filter of free-surface fields
  prism    -- prisms over an unstructured triangular surface mesh: operator,
              Laplace solve, w
"""
from . import filter, gll, mesh, operator, prism, solve, surface, tlm  # noqa: F401
