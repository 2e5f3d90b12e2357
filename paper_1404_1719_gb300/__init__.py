"""GB300-native (sm_103a) pair-process neutrino rate kernel for ray-by-ray transport.

The e+e- <-> nu nubar kernel Phi_l(eps, eps'), l = 0, 1, evaluated for every radial zone of every
ray and contracted with the zone's partner spectra into emissivities and opacities, with T / eta_e
tangents for the implicit transport Newton solve (Marek et al., arXiv:1404.1719, sec. 2.1-2.2, 4).
The per-ray Newton systems those tangents feed are solved by the batched block-tridiagonal solver
(sec. 2.1). All arithmetic runs in the CUDA library libvx_rates.so (C ABI: include/vx_rates.h,
include/vx_btd.h); this package is the ctypes binding and PyTorch wrappers that supply device
memory and streams.
"""
from . import capi
from ._build import build
from .btd import BlockTridiagSolver
from .rates import PairRates, VxRatesFn

__all__ = ["capi", "build", "BlockTridiagSolver", "PairRates", "VxRatesFn"]
