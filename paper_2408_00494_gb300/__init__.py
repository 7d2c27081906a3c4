"""GB300 (sm_103a) implementation of the BSS-MPPI hot path behind a C ABI (include/bssmppi.h).

``bssmppi`` is the thin ctypes binding of libbssmppi.so; ``_build`` compiles it in-tree with nvcc.
"""
from . import _build  # noqa: F401
