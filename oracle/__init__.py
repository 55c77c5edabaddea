"""Plain, slow FP64 CPU oracle for the nodal DG Maxwell hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only the tests, `__graft_entry__.smoke()` and the benchmark's
CPU-baseline leg (`bench.py`) may use it.  It shares no code with the CUDA
library (paper_0901_1024_gb300/): different polynomial basis, different
quadrature, different face matching, different geometry formulas.

What it computes (Kloeckner, Warburton, Bridge, Hesthaven, "Nodal
Discontinuous Galerkin Methods on Graphics Processors"):
  * refelem  -- interpolation nodes, Lagrange-basis mass / differentiation /
                face-mass / lifting matrices (Section 2, Eq. dg-global-matrices,
                Fig. lifting-matrix), written from their integral definitions.
  * mesh     -- per-element affine maps, metric terms, outward normals, face
                scalings and face-node connectivity (Section 2, Eq.
                dg-reference-matrices; face index lists of Section 5.2).
  * maxwell  -- the semi-discrete right-hand side for Maxwell's equations with
                the upwind flux and PEC walls (Eq. semidiscrete-dg, Section 6),
                the LSERK4 time stepper and the discrete energy.

Every function is pinned by `-m "not gpu"` tests against closed forms
(monomial exactness, exact integrals, summation by parts, geometric
identities, energy identities, the exact cavity eigenmode).
"""
from .refelem import RefElement, ref_element  # noqa: F401
from .mesh import Mesh, build_mesh  # noqa: F401
from .maxwell import (  # noqa: F401
    rhs, lserk4_coefficients, lserk4_run, energy, cfl_dt, stage_update,
)
