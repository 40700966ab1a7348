"""GB300-native nested-grid lattice Boltzmann hot path (D3Q19 MRT-LES and
D3Q27 factorized cascaded collision with Yu-style time nesting).

The compute lives in the CUDA library ``liblbm.so`` (C ABI in include/lbm.h);
``paper_1206_0389_gb300.lbm`` is its thin ctypes binding.  Importing the
binding fails loudly when the library has not been built: there is no CPU
fallback.
"""
from .lbm import *  # noqa: F401,F403
