"""GB300 (sm_103a) continuous-component normal integration (arXiv 2510.11508).

The compute path is libni (CUDA kernels behind the C ABI in include/ni.h); the
Python module `paper_2510_11508_gb300.ni` is its ctypes binding.
"""
__all__ = ["ni", "build"]
