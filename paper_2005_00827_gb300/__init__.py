"""GB300-native quasi-particle fRG flow library (Rohe & Honerkamp, arXiv:2005.00827).

The compute path is the C-ABI shared library built from ``csrc/`` for sm_103a;
``api`` holds the thin ctypes binding with the same call names as
``include/qpfrg.h``.  Importing the package does not load the library; the
first API call does, and fails loudly when the CUDA build is missing.
"""
