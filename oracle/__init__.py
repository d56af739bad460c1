"""FP64 CPU oracle for the elastance and mobility Nystrom/GMRES hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or calls this package; only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA path: it assembles the dense Nystrom matrix of
the paper's second-kind equations and solves it by LU, in float64, with plain
numpy/scipy, so that each step can be checked against the paper by eye.

Discretisation (a reading, the paper uses Gauss-Legendre panels with GLQBX
quadrature): each boundary is sampled at equispaced parameter values and the
periodic trapezoidal rule is the Nystrom quadrature.  Both kernels K (Laplace,
target normal) and the Stokes traction kernel are smooth on smooth curves; the
diagonal entries are their limits, -kappa/(4 pi) and -(kappa/(2 pi)) tau tau^T.

Modules:
  geometry  -- weights, normals, curvature, per-body length/centroid/W (Sec. 3, 4.1)
  laplace   -- elastance: K, L, sigma, RHS, LU solve, potentials (Sec. 3)
  stokes    -- mobility: stresslet traction kernel, L, rho, LU solve, v/omega (Sec. 4)
  capacitance -- the capacitance problem (potentials -> charges) by a different
               integral equation, for the paper's round trip (Sec. 6.1)
  resistance  -- the resistance problem (rigid motions -> forces and torques) by
               a different integral equation, for the mobility round trip (Sec. 6.2)

Every function here is pinned by tests against closed forms, the paper's
identities and the paper's printed two-disc values (see tests/test_oracle_pins.py).
"""
from . import capacitance, geometry, laplace, resistance, stokes  # noqa: F401
