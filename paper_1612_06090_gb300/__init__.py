"""GB300-native SPH density / smoothing-length solver (arXiv:1612.06090 hot path).

The compute lives in hand-written sm_103a CUDA behind a C ABI (``include/sph.h``,
``libsph.so``).  ``binding`` loads that library through ctypes; ``inputs`` draws the
seeded synthetic particle sets.  Importing the package loads nothing: the CUDA library
is opened on first use of the binding and fails loudly when it is missing.
"""
__all__ = ["binding", "inputs", "build"]
