"""GB300-native super-potential GS/FFT solver for the 3D free-space Poisson equation
(Exl & Schaffer, arXiv:2506.04489).

``Plan`` wraps the C ABI of ``include/superpot.h``; PyTorch supplies device memory and
streams.  The CUDA library is loaded on first use of ``Plan`` and its absence is an
error (there is no CPU path).  ``workloads`` holds the seeded input densities.
"""
from .plan import Plan, precision_dtype  # noqa: F401

__all__ = ["Plan", "precision_dtype"]
