"""GB300-native two-population compressible lattice Boltzmann (arXiv:2102.09512).

The compute path is the CUDA library ``libelbm.so`` (sources in ``csrc/``), reached
through the thin ctypes binding in :mod:`paper_2102_09512_gb300.elbm`.  Importing
this package loads nothing; the binding loads the library on first use and raises
if it has not been built.
"""
__all__ = ["cases", "elbm"]
