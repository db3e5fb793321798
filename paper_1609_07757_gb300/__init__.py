"""GB300-native Integral-Screened CI sigma step (arXiv:1609.07757).

The compute path is the CUDA library libiscsi.so (C ABI in include/iscsi.h);
``paper_1609_07757_gb300._lib`` is its ctypes binding with the C names, and
``synthetic`` holds the seeded input generator.  Importing the package loads
nothing; the first binding call builds (if needed) and loads the library.
"""
__all__ = ["_lib", "synthetic"]
