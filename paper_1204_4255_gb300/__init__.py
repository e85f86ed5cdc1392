"""GB300 (sm_103a) RK4IP for coupled stochastic PDEs on periodic Fourier lattices.

The compute lives in ``libxsde.so`` (hand-written CUDA kernels behind the C-ABI
of ``include/xsde.h``); ``xsde`` is its thin ctypes binding.  Build the library
with ``paper_1204_4255_gb300.build.build()``.
"""
from . import xsde  # noqa: F401
from .xsde import Problem, XsdeError  # noqa: F401

__all__ = ["xsde", "Problem", "XsdeError"]
