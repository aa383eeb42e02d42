"""GB300-native axisymmetric lattice Boltzmann solver (arXiv:1003.0282).

The compute path is the C-ABI library ``libaxlbm`` (hand-written CUDA for
sm_103a) declared in ``include/axlbm.h``; :mod:`paper_1003_0282_gb300.axlbm`
is its thin ctypes binding.  Importing this package loads nothing native; the
binding loads the library on first use and raises if it is missing.
"""
__all__ = ["inputs"]
