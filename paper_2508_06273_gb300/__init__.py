"""GB300-native (sm_103a) fully discrete third-order Active Flux method for
the 2D Euler equations (Chudzik, Helzel, Porfetye, arXiv 2508.06273).

The numerical work runs in hand-written CUDA kernels behind the C ABI
declared in ``include/af.h``; ``paper_2508_06273_gb300.af`` is a thin ctypes
binding of that library.  Importing the package does not load the library;
the first call into ``af`` does, and fails loudly if it is missing.
"""
__all__ = ["af", "workloads"]
