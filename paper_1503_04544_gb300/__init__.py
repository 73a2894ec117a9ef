"""GB300-native cut-cell discrete-velocity BGK solver (arXiv:1503.04544).

The compute path is the CUDA library ``libdvm.so`` (sources in ``csrc/``),
reached through the ctypes binding in :mod:`paper_1503_04544_gb300.dvm`.
Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
