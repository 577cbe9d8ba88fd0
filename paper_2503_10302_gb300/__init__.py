"""GB300-native p-bit Monte Carlo for 3D +-J spin glasses (arXiv 2503.10302).

The compute path is the CUDA library libpcomp.so (C ABI in include/pcomp.h);
``pcomp`` is its ctypes binding and ``workloads`` the seeded input generators.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "pcomp", "build"]
