"""GB300-native reserves for non-unit-linked life policies.

The vector reserve recurrence of Tucker & Bull (arXiv 1401.1757, Eq.
generalForm) for every policy x scenario, as hand-written sm_103a CUDA kernels
behind the C ABI in include/rsv.h.  ``rsv`` is the ctypes binding (same names
as the C functions); the library is built in-tree by ``_build.build_library``.
"""
from . import rsv  # noqa: F401
from .rsv import *  # noqa: F401,F403
