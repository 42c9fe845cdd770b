"""FP64 CPU oracle of the implicit spectral/hp DG compressible Navier-Stokes
method (JFNK + restarted GMRES + block-relaxed Jacobi + Newton + SDIRK).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library and never imports it: it is a plain, slow, per-element dense
restatement of the method, written so that each step can be checked against
the paper by eye.  Its inputs (meshes, parameters, seeded random vectors) come
from the separate `workloads` package.

Modules
  basis     1-D Gauss-Legendre rule, modified (Karniadakis-Sherwin) and nodal
            bases, tensor-product tables                         (Sec. 3.1)
  geometry  isoparametric map, metrics, face normals and surface Jacobians
  physics   Euler/viscous fluxes, Roe and HLLC fluxes, analytic fields,
            manufactured forcing, boundary states              (Sec. 2, 3.1)
  dg        the residual R(u) = M^-1 L(u, t) of the matrix form    (Sec. 3.1)
  implicit  JFNK product, GMRES, BRJ preconditioner, Newton, SDIRK
                                                     (Sec. 3.2, Sec. 4.2.2)

Parity status: every function is pinned by a CPU test (tests/test_oracle_*.py)
except where its docstring says "parity unpinned".
"""
from .basis import (gauss_legendre, jacobi, modified_basis, gll_points,  # noqa: F401
                    lagrange_basis, tensor_tables)
from .dg import DG  # noqa: F401
from .implicit import (jvp, gmres, BRJ, newton, sdirk_step, sdirk_tableau, bdf2_step,  # noqa: F401
                       NewtonConfig, GmresConfig)
