"""GB300-native MPCD solvent collision-interval update (RMPCDMD method, arXiv:1608.04904).

The compute path is the CUDA library built from ``csrc/`` (sm_103a) behind the
C ABI declared in ``include/rmpcd.h``; ``api`` is a thin ctypes binding to it.
"""
