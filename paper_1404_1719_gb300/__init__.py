"""GB300-native (sm_103a) pair-process neutrino rate kernel for ray-by-ray transport.

The e+e- <-> nu nubar kernel Phi_l(eps, eps'), l = 0, 1, evaluated for every radial zone of every
ray and contracted with the zone's partner spectra into emissivities and opacities, with T / eta_e
tangents for the implicit transport Newton solve (Marek et al., arXiv:1404.1719, sec. 2.1-2.2, 4).
All arithmetic runs in the CUDA library libvx_rates.so (C ABI: include/vx_rates.h); this package
is the ctypes binding and a PyTorch wrapper that supplies device memory and streams.
"""
from . import capi
from ._build import build
from .rates import PairRates, VxRatesFn

__all__ = ["capi", "build", "PairRates", "VxRatesFn"]
