"""GB300-native Canny edge detector (sm_103a CUDA kernels behind a C ABI).

The native library is loaded lazily by :mod:`paper_1710_07745_gb300.canny`;
importing this package alone loads nothing.
"""
__all__ = ["canny", "synth"]
