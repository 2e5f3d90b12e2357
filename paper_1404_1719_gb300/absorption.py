"""PyTorch-facing wrapper of the charged-current absorption and emission rates on free nucleons
(include/vx_abs.h): device buffers and streams come from torch, every step runs in libvx_rates.

    ab = AbsRates(eps)                        # nu_e n <-> e- p, anti-nu_e p <-> e+ n
    out = ab.evaluate(state)                  # j0, chi0, j1, chi1 [Z][S][N] (j1 = chi1 = 0)
    res = ab.adjoint(state, forward=True)     # jac [Z][S][N][4][3] d/d(T, eta_e, Y_e) and the rates
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi
from .rates import _OUT_KEYS, PairRates, _ptr


class AbsRates(PairRates):
    """Handle of the absorption and emission rates for one energy grid and species list;
    precision "mixed" (FP32 occupation factors, FP64 prefactors) or "fp64". Only the zone state is
    read: the rates do not depend on the neutrino spectra."""

    def __init__(self, eps, species=(0, 1, 2), g2: float = 1.0, precision: str = "mixed", device=None):
        self.eps = np.ascontiguousarray(eps, dtype=np.float64)
        self.species = np.ascontiguousarray(species, dtype=np.int32)
        self.N, self.S = len(self.eps), len(self.species)
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
        prec = {"mixed": capi.VX_PREC_MIXED, "fp64": capi.VX_PREC_FP64}[precision]
        cfg = capi.vx_config(
            n_bins=self.N, eps=self.eps.ctypes.data_as(capi._dp), weights=None, n_mu=0, n_e=0,
            n_species=self.S, species=self.species.ctypes.data_as(capi._ip), sin2w=0.0, g2=g2, norm=1.0,
            eta_fp64=0.0, prec=prec, flags=0)
        with torch.cuda.device(self.device):
            self._h = capi.vx_abs_create(cfg)

    def close(self):
        if getattr(self, "_h", None):
            capi.vx_abs_destroy(self._h)
            self._h = None

    def entries_per_zone(self) -> int:
        return self.S * self.N

    def _state_batch(self, state, ray_offsets, stream):
        Z = state.shape[0]
        if (not torch.is_tensor(state) or state.dtype != torch.float64 or not state.is_cuda or not state.is_contiguous()
                or tuple(state.shape) != (Z, 4)):
            raise ValueError(f"state must be a contiguous CUDA float64 tensor of shape {(Z, 4)}")
        if state.device != self.device:
            raise ValueError(f"state is on {state.device}, the handle on {self.device}")
        offs, nr = self._offsets(ray_offsets, Z, stream)
        b = capi.vx_batch(n_rays=nr, n_zones=Z, ray_offsets=None if offs is None else ctypes.cast(offs.data_ptr(), capi._ip),
                          state=state.data_ptr(), J=None, H=None)
        b._keep = offs
        return b

    def evaluate(self, state, J=None, H=None, ray_offsets=None, out=None, stream=None) -> dict:
        """Rates j0, chi0, j1, chi1 ([Z][S][N] float64). J and H are accepted for the common
        signature and not read."""
        Z = state.shape[0]
        b = self._state_batch(state, ray_offsets, stream)
        if out is not None:
            for k in _OUT_KEYS:
                self._check_out(f"out[{k!r}]", out.get(k), (Z, self.S, self.N))
        res = out if out is not None else self._alloc(Z)
        o = capi.vx_out(*(_ptr(res[k]) for k in _OUT_KEYS), None)
        capi.vx_abs_eval(self._h, b, o, self._stream(stream))
        return res

    def adjoint(self, state, J=None, H=None, grad_out=None, jacobian: bool = True, forward: bool = False,
                ray_offsets=None, stream=None) -> dict:
        """Jacobian [Z][S][N][4][3] (d/dT at fixed eta_e, Y_e, rho; d/deta_e; d/dY_e) and, with
        forward=True, the rates of the same pass. Every rate is proportional to rho, so its
        derivative in rho is rate / rho."""
        if grad_out is not None or not jacobian:
            raise ValueError("the absorption rates return the full Jacobian (no vector-Jacobian product)")
        Z = state.shape[0]
        b = self._state_batch(state, ray_offsets, stream)
        res = {"jac": torch.empty((Z, self.S, self.N, 4, 3), dtype=torch.float64, device=self.device)}
        fwd = None
        if forward:
            res.update(self._alloc(Z))
            fwd = capi.vx_out(*(_ptr(res[k]) for k in _OUT_KEYS), None)
        capi.vx_abs_adjoint(self._h, b, res["jac"].data_ptr(), fwd, self._stream(stream))
        return res

    def spectral(self, *a, **k):
        raise NotImplementedError("the absorption rates do not depend on the neutrino spectra")

    def check(self, stream=None) -> bool:
        return capi.vx_abs_check(self._h, self._stream(stream)) == capi.VX_OK
