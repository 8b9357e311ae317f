"""FP64 CPU oracle for the mass-lumped KMV acoustic FWI hot path.

This package is TEST INFRASTRUCTURE. It is a plain, slow, FP64 restatement of what the
paper's method computes: KMV reference elements, global lumped mass, stiffness and damping
layer operators, the leapfrog time step of Eq. (forward3), the discrete adjoint (the
transposed recurrence of Section 3.5), and the mesh-independent gradient of Eq.
(gradient3). Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it. The product path (the CUDA
library and its Python binding) never imports, calls or links anything here, and this
package imports nothing from the product.

Modules:
  kmv       reference elements (nodes, lumping weights, nodal basis, derivative matrices)
  mesh      DoF numbering by node position, affine geometry, point location
  assemble  global sparse operators of Appendix A
  wave      forward / adjoint / gradient recurrences (Eqs. forward3, acoustic_pml_FEM_adj,
            gradient3), misfit (Eq. l2error), CFL estimate (Eq. spectral)
  analytic  Ricker wavelet and the 2D free-space Green's function image sum

Parity status: every function is pinned by tests under tests/test_oracle_*.py. The
KMV4tri/KMV5tri nodes (not printed in the paper; solved here from the moment equations at
degree k + k' - 2) are pinned by their convergence order, not by a table. The
damping-layer time scheme (the printed block matrices are garbled; see wave.py) is "parity
unpinned" against the paper's exact scheme.
"""
