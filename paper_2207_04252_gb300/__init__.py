"""GB300-native hot path of the RoSSBi3D method (arXiv:2207.04252).

librossbi.so (csrc/, C ABI in include/rossbi.h) holds the CUDA kernels and
host runtime; ``rossbi`` is its ctypes binding and ``workloads`` builds grids
and initial states for the synthetic workloads.
"""
from . import rossbi  # noqa: F401
