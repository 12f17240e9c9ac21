"""GB300 implementation of the IPM hot path (Kusch, Wolters, Frank, arXiv:1912.09238).

The compute path is libipm.so (CUDA C++ for sm_103a, C ABI in include/ipm.h); ``ipm`` is its
ctypes binding and ``workloads`` holds the parameters of the benchmark workloads.
"""
from . import ipm, workloads  # noqa: F401
