"""GB300 (sm_103a) library for the scale-invariant binary MERA of
arXiv:1906.12030: ascending/descending superoperators, the scale-invariant
fixed point, the u/w environments, the polar update, the energy and the
optimisation sweep, behind a C ABI (``include/mera.h``).

This Python package is a thin ctypes binding with the same names as the C
entry points; PyTorch supplies device memory and streams.  Every step of the
computation runs in the library's CUDA kernels; there is no CPU fallback.
"""
from .api import *  # noqa: F401,F403
from .api import __all__  # noqa: F401
