"""GB300-native generalized Poisson / Poisson-Boltzmann PCG solver.

The compute path is the CUDA library libgps.so (C ABI in include/gps.h);
``gps`` is its thin ctypes binding and ``build`` compiles it for sm_103a.
"""
from . import build  # noqa: F401

__all__ = ["build", "gps"]
