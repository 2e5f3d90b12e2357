"""GB300-native (sm_103a) neutrino interaction-rate kernels for ray-by-ray transport.

The e+e- <-> nu nubar pair kernel Phi_l(eps, eps'), l = 0, 1, evaluated for every radial zone of
every ray and contracted with the zone's partner spectra into emissivities and opacities, with
T / eta_e tangents for the implicit transport Newton solve (Marek et al., arXiv:1404.1719,
sec. 2.1-2.2, 4); the same for inelastic neutrino-electron scattering; the charged-current
absorption and emission rates on free nucleons; the electron-gas closure eta_e(rho, Y_e, T) and
its chain rule; and the batched block-tridiagonal solver of the per-ray Newton systems
(sec. 2.1). All arithmetic runs in the CUDA library libvx_rates.so (C ABI: include/vx_rates.h,
vx_nes.h, vx_abs.h, vx_eos.h, vx_btd.h, vx_probe.h); this package is the ctypes binding and
PyTorch wrappers that supply device memory and streams.
"""
from . import capi
from ._build import build
from .absorption import AbsRates
from .btd import BlockTridiagSolver
from .nes import NesRates, eos_chain, eos_eta
from .rates import PairRates, VxRatesFn

__all__ = ["capi", "build", "AbsRates", "BlockTridiagSolver", "NesRates", "PairRates", "VxRatesFn", "eos_chain", "eos_eta"]
