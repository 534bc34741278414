"""GB300-native (sm_103a) one-step Lagrange-Remap library (DirectCF remap,
VOF/PLIC material fluxes) after Chaudet, arXiv 2208.13409.

The compute path is the CUDA library built from ``csrc/`` behind the C ABI
declared in ``include/lr.h``; ``lr`` is its thin ctypes binding.  Importing
this package does not load the library: ``lr.load()`` does, and fails loudly
when it is missing.
"""
__all__ = ["lr", "problems"]
