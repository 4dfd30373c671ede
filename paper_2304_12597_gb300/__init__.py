"""GB300 (sm_103a) implementation of the new ParaDiag method (arXiv 2304.12597).

The compute path is the CUDA library built from csrc/ (C ABI in
include/paradiag.h); this package only marshals arguments.  Importing it loads
the library and raises if it has not been built: there is no CPU fallback.
"""
from . import _binding  # noqa: F401
from ._binding import (  # noqa: F401
    PD_FP64,
    PD_MIXED,
    ParadiagError,
    paradiag_destroy,
    paradiag_dst_y,
    paradiag_kernel_times,
    paradiag_last_vectors,
    paradiag_plan,
    paradiag_set_timing,
    paradiag_shifted_solve,
    paradiag_solve,
    paradiag_solve_host,
    paradiag_time_dft,
    paradiag_time_idft,
    paradiag_version,
    paradiag_workspace_size,
)
from .plan import Plan  # noqa: F401

_binding.load()
