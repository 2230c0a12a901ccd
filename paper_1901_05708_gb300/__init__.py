"""GB300-native matrix-profile sweep (AAMP / p-norm / ACAMP, arXiv:1901.05708).

The compute path is the CUDA library ``libmp.so`` built from ``csrc/``; this
package only marshals arguments to its C ABI (``include/mp.h``).  Importing
the package loads nothing; the library is opened on first use and a missing
or unloadable library raises immediately (there is no CPU fallback).
"""
__all__ = ["workloads"]
