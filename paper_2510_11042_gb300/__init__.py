"""GB300-native lattice-Boltzmann electromagnetic scattering (arXiv 2510.11042).

The product is the C-ABI CUDA library built from csrc/ (include/lbem.h); the
Python module ``lbem`` is its thin ctypes binding.  Importing this package does
not load the library; ``lbem.lib()`` does, and fails loudly when it is missing.
"""
__all__ = ["lbem", "build"]
