"""GB300-native projective-integration PIC (Cazeaux & Hesthaven, arXiv:1610.01071).

The compute path is the CUDA library ``libpepic.so`` built from ``csrc/``; the
Python side only marshals arguments to its C ABI (``include/pepic.h``).
"""
