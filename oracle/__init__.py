"""Plain FP64 CPU oracle (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline / reference leg may
import this package.  The CUDA library and its Python binding never do, and the
two share no code.  See oracle/helmholtz.py for the functions and their citations.
"""
from . import helmholtz, dense  # noqa: F401
