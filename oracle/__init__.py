"""FP64 CPU oracle for arXiv 2304.12597's ParaDiag (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The CUDA path never does; it fails loudly instead.
"""
from . import native, reference  # noqa: F401
