"""GB300-native axisymmetric Allen-Cahn phase-field MRT lattice Boltzmann library.

The compute path is the CUDA shared library ``libaxilbm.so`` (sm_103a) behind
the C ABI declared in ``include/lbm.h``; ``lbm`` is its ctypes binding.  The
library is loaded lazily so that host-only modules (``workloads``) import
without a GPU.
"""
__all__ = ["lbm", "workloads"]
