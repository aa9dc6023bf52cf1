"""GB300-native FD-CGKS hot path (sm_103a CUDA kernels behind a C ABI).

The CUDA library is loaded lazily by :mod:`paper_2606_17772_gb300.fdcgks`;
importing the package itself loads nothing.
"""
