"""PyTorch-facing wrappers of the NES rate kernel (include/vx_nes.h) and of the electron-gas
closure (include/vx_eos.h): device buffers and streams come from torch, every step runs in
libvx_rates.

    nes = NesRates(eps, n_mu=16, n_e=48)                 # inelastic nu-e scattering
    out = nes.evaluate(state, J, H)                       # j0, chi0, j1, chi1 [Z][S][N]
    jac = nes.jacobian(state, J, H)                       # [Z][S][N][4][3] d/d(T, eta_e, Y_e)
    deta = eos_eta(state)                                 # fills state[:, 1], returns d eta/d(T, Y_e, rho)
    jac_rho = eos_chain(jac, deta)                        # d/d(T, Y_e, rho) at fixed (rho, Y_e), ...
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi
from .rates import _OUT_KEYS, PairRates, _ptr


class NesRates(PairRates):
    """Handle of the NES kernel for one energy grid and quadrature (n_e a multiple of 3: three
    electron-energy panels of n_e/3 nodes). precision "mixed" or "fp64"."""

    def __init__(self, eps, n_mu: int, n_e: int, species=(0, 1, 2), weights=None, sin2w: float = 0.23,
                 g2: float = 1.0, norm: float = 1.0, precision: str = "mixed", device=None):
        self.eps = np.ascontiguousarray(eps, dtype=np.float64)
        self.weights = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
        self.species = np.ascontiguousarray(species, dtype=np.int32)
        self.N, self.S = len(self.eps), len(self.species)
        self.n_mu, self.n_e = int(n_mu), int(n_e)
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
        prec = {"mixed": capi.VX_PREC_MIXED, "fp64": capi.VX_PREC_FP64}[precision]
        cfg = capi.vx_config(
            n_bins=self.N, eps=self.eps.ctypes.data_as(capi._dp),
            weights=None if self.weights is None else self.weights.ctypes.data_as(capi._dp),
            n_mu=self.n_mu, n_e=self.n_e, n_species=self.S, species=self.species.ctypes.data_as(capi._ip),
            sin2w=sin2w, g2=g2, norm=norm, eta_fp64=0.0, prec=prec, flags=0)
        with torch.cuda.device(self.device):
            self._h = capi.vx_nes_create(cfg)

    def close(self):
        if getattr(self, "_h", None):
            capi.vx_nes_destroy(self._h)
            self._h = None

    def entries_per_zone(self) -> int:
        return self.N * self.N

    def evaluate(self, state, J, H, ray_offsets=None, phi: bool = False, out=None, stream=None) -> dict:
        """Rates j0, chi0, j1, chi1 ([Z][S][N] float64); phi=True adds the kernel dump
        [Z][2 X][2 dir][2 l][N][N] (dir 0 = in, 1 = out)."""
        Z = state.shape[0]
        b = self._batch(state, J, H, ray_offsets, stream)
        if out is not None:
            for k in _OUT_KEYS:
                self._check_out(f"out[{k!r}]", out.get(k), (Z, self.S, self.N))
        res = out if out is not None else self._alloc(Z)
        if phi and "phi" not in res:
            res["phi"] = torch.empty((Z, 2, 2, 2, self.N, self.N), dtype=torch.float64, device=self.device)
        o = capi.vx_out(*(_ptr(res[k]) for k in _OUT_KEYS), _ptr(res.get("phi")) if phi else None)
        capi.vx_nes_eval(self._h, b, o, self._stream(stream))
        return res

    def adjoint(self, state, J, H, grad_out=None, jacobian: bool = True, forward: bool = False,
                ray_offsets=None, stream=None) -> dict:
        """Jacobian [Z][S][N][4][3] and, with forward=True, the rates of the same pass."""
        if grad_out is not None or not jacobian:
            raise ValueError("the NES kernel returns the full Jacobian (no vector-Jacobian product)")
        Z = state.shape[0]
        b = self._batch(state, J, H, ray_offsets, stream)
        res = {"jac": torch.empty((Z, self.S, self.N, 4, 3), dtype=torch.float64, device=self.device)}
        fwd = None
        if forward:
            res.update(self._alloc(Z))
            fwd = capi.vx_out(*(_ptr(res[k]) for k in _OUT_KEYS), None)
        capi.vx_nes_adjoint(self._h, b, res["jac"].data_ptr(), fwd, self._stream(stream))
        return res

    def evaluate_host(self, state, J, H, ray_offsets=None, out=None) -> dict:
        """End-to-end call on host arrays (numpy or pinned torch CPU tensors): vx_nes_eval_host
        copies chunks of zones in, evaluates and copies the rates back, overlapping the copies of
        one chunk with the kernel of the next. Returns host tensors (pinned unless `out` given)."""
        b, Z = self._host_batch(state, J, H, ray_offsets)
        res, o = self._host_out(Z, out)
        with torch.cuda.device(self.device):
            capi.vx_nes_eval_host(self._h, b, o)
        return res

    def adjoint_host(self, state, J, H, forward: bool = True, ray_offsets=None, out=None, jac=None) -> dict:
        """End-to-end rates and Jacobian on host arrays (vx_nes_adjoint_host)."""
        b, Z = self._host_batch(state, J, H, ray_offsets)
        res, o = self._host_out(Z, out) if forward else ({}, None)
        if jac is not None:
            self._check_out("jac", jac, (Z, self.S, self.N, 4, 3), host=True)
        res["jac"] = jac if jac is not None else torch.empty((Z, self.S, self.N, 4, 3), dtype=torch.float64,
                                                             pin_memory=True)
        with torch.cuda.device(self.device):
            capi.vx_nes_adjoint_host(self._h, b, res["jac"].data_ptr(), o)
        return res

    def spectral(self, *a, **k):
        raise NotImplementedError("spectral derivatives are provided for the pair kernel")

    def spectral_host(self, *a, **k):
        raise NotImplementedError("spectral derivatives are provided for the pair kernel")

    def check(self, stream=None) -> bool:
        return capi.vx_nes_check(self._h, self._stream(stream)) == capi.VX_OK


def _dev_f64(t, name, shape=None):
    if not (torch.is_tensor(t) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}")


def eos_eta(state, stream=None):
    """Fills state[:, 1] (eta_e) from T, Y_e, rho by the massless electron-gas closure; returns
    d eta_e / d(T, Y_e, rho) [Z][3]."""
    _dev_f64(state, "state")
    if state.dim() != 2 or state.shape[1] != 4:
        raise ValueError("state must be [Z][4]")
    Z = state.shape[0]
    deta = torch.empty((Z, 3), dtype=torch.float64, device=state.device)
    s = (stream or torch.cuda.current_stream(state.device)).cuda_stream
    capi.vx_eos_eta(Z, state.data_ptr(), deta.data_ptr(), s)
    return deta


def eos_chain(jac, deta, out=None, stream=None):
    """Derivatives at fixed (rho, Y_e) from a kernel Jacobian [Z][..][3] (d/dT at fixed eta, d/deta,
    d/dY_e at fixed eta): returns [Z][..][3] = (d/dT, d/dY_e, d/drho). A rate with its own
    dependence on rho at fixed eta (the absorption rates: rate / rho) needs that term added."""
    _dev_f64(jac, "jac")
    _dev_f64(deta, "deta", (jac.shape[0], 3))
    if jac.shape[-1] != 3:
        raise ValueError("the last axis of jac must hold the 3 inputs")
    Z = jac.shape[0]
    rows = jac.numel() // (3 * max(Z, 1)) if Z else 0
    res = torch.empty_like(jac) if out is None else out
    _dev_f64(res, "out", jac.shape)
    s = (stream or torch.cuda.current_stream(jac.device)).cuda_stream
    capi.vx_eos_chain(Z, rows, deta.data_ptr(), jac.data_ptr(), res.data_ptr(), s)
    return res
