"""GB300-native structured FISTA (sFISTA) for Tikhonov image deblurring.

Chen, Nagy, Xi, Yu, "Structured FISTA for Image Restoration" (arXiv
1901.00913): the blur is approximated by a short Kronecker sum
sum_i A_i kron B_i (Sec. 2) and Alg. 2 runs FISTA on the matrix model
min 0.5||sum_i B_i X A_i^T - B||_F^2 + 0.5 lambda^2 ||X||_F^2.

The compute lives in ``libsfista.so`` (C ABI, ``include/sfista.h``): FP64 host
setup, and sm_103a CUDA kernels for the operator and the fused FISTA
epilogue.  ``api`` is the ctypes binding; ``workloads`` makes seeded
synthetic inputs; ``build`` compiles the library in-tree.
"""
from . import api  # noqa: F401
from .api import Sfista, SfistaError  # noqa: F401
