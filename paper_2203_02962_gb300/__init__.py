"""fehom: a GB300-native FFT-preconditioned matrix-free FE homogenization solver.

The package holds the ctypes binding to the C-ABI library ``libfehom.so`` (``fehom``) and the
seeded synthetic input generators (``inputs``).  Importing the package loads nothing; the CUDA
library is loaded on first use of :mod:`paper_2203_02962_gb300.fehom`.
"""
