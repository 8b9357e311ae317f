"""GB300 library for the explicit mass-lumped KMV acoustic time step of time-domain full
waveform inversion (arXiv 2108.10946): forward solve, discrete adjoint and mesh-independent
gradient on triangles (k = 2..5) and tetrahedra (k = 2, 3), as hand-written sm_103a CUDA
behind the C ABI of include/fwi.h. This package is the ctypes binding of that library."""
from ._build import build  # noqa: F401
from .lib import Batch, FwiError, Mesh, launch_count, load  # noqa: F401
