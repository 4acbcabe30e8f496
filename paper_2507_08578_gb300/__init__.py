"""GB300-native plane-wave Kohn-Sham Hamiltonian application and Chebyshev-filtered eigensolver.

The compute path is the CUDA library ``libkss.so`` (sources in ``csrc/``, C ABI in
``include/kss.h``); ``kss`` is its ctypes binding.  Build it with ``build.build()``.
"""
from . import kss  # noqa: F401
from .kss import KssError  # noqa: F401
