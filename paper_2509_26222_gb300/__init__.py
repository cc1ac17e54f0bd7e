"""GB300-native RBF terrain library: evaluation of the terrain model, the
recursive ridge update of its weights and the soft-constraint cost
(arXiv 2509.26222, Sec. III-V), as CUDA kernels behind a C ABI
(include/rbfgb.h, librbfgb.so).

``native`` is the ctypes binding; ``workloads`` holds the seeded synthetic
inputs.  Importing the package does not load the library; ``native.load()``
does, and raises if it was not built.
"""
from . import build, workloads  # noqa: F401

__all__ = ["build", "workloads", "native"]
