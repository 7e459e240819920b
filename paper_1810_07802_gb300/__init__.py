"""GB300-native phase-field DUGKS (arXiv:1810.07802): CUDA kernels for sm_103a
behind a C ABI (include/dugks.h), with a thin ctypes binding.

Importing the package loads nothing; `paper_1810_07802_gb300.solver` loads the
CUDA library and fails loudly if it has not been built.
"""
__all__ = ["workloads"]
