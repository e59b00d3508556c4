"""GB300-native (sm_103a) forward and adjoint harmonic radiance Monte Carlo.

Hochuli, Powell, Arridge & Cox, "Quantitative photoacoustic tomography using forward and
adjoint Monte Carlo models of radiance" (arXiv 1608.05238).  The compute path is the CUDA
library libmcr.so (C ABI in include/mcr.h); :mod:`.mcr` is its thin binding.  Importing the
package loads nothing: the library is loaded on first use and its absence is an error.
"""
__all__ = ["mcr", "workloads"]
