"""TEST INFRASTRUCTURE: the FP64 CPU oracle for surrogate IGA stiffness assembly.

Plain, slow and written to be checked by eye against Drzisga, Keith &
Wohlmuth, "The surrogate matrix methodology: low-cost assembly for
isogeometric analysis".  The exact Gauss-quadrature rows come from the plain-C
routine in ``iga_oracle.c``; the surrogate steps (sampling lattice, stencil
samples, per-offset B-spline interpolation, symmetric copy, kernel-preserving
diagonal) and the stencil SpMV / CG are numpy in ``surrogate.py`` and
``linalg.py``; the variant with per-offset interpolation domains is
``per_offset.py``.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path (``paper_1904_06971_gb300``) and neither imports the
other.
"""
from ._lib import build, num_threads  # noqa: F401
from .surrogate import (  # noqa: F401
    offsets, center_slot, multi_index, flat_index, exact_rows, exact_matrix, elementwise_dense,
    ell_to_dense, omega_box, sample_indices, interp_knots, bspline_basis,
    SurrogateSetup, surrogate_setup, surrogate_rows, surrogate_matrix,
    gauss_legendre, open_uniform_knots, bspline_all, coefficient, geometry_map,
)
from .linalg import apply, interior_dofs, cg, relative_entry_error  # noqa: F401
from . import per_offset, adjoint, mass, manufactured  # noqa: F401
