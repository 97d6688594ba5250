"""GB300-native MacLAB: the macroscopic lattice Boltzmann time step in CUDA for sm_103a.

The compute path is the C-ABI library ``libmaclab.so`` (hand-written CUDA,
declared in ``include/maclab.h``); ``maclab.py`` is a thin ctypes binding with
the same names.  Importing this package does not load the library; the first
call that needs it does, and fails loudly if it has not been built
(``paper_1901_02716_gb300._build.build()``).
"""
from . import inputs  # noqa: F401  (pure numpy, no GPU)

__all__ = ["inputs", "maclab"]
