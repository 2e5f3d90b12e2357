"""PyTorch-facing wrapper of the C ABI: device buffers and streams come from torch, every step of
the computation runs in libvx_rates.

    rates = PairRates(eps, n_mu=32, n_e=64)                    # one handle per device/stream
    out = rates.evaluate(state, J, H)                           # dict of [Z][S][N] float64 tensors
    jac = rates.jacobian(state, J, H)                           # [Z][S][N][4][3]
    blk = rates.spectral(state, J, H)["blocks"]                 # [Z][S][4][N][N], d rates / d(J, H)
    j0, chi0, j1, chi1 = VxRatesFn.apply(rates, state, J, H)    # differentiable in state, J and H
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi

_OUT_KEYS = ("j0", "chi0", "j1", "chi1")


def _ptr(t):
    return None if t is None else t.data_ptr()


class PairRates:
    """Handle of the pair-process rate library for one energy grid and quadrature (split=True:
    the split discrete rule in electron energy, panels meeting at the Fermi edge; precise=True:
    the precise mode, VX_PRECISE, for results whose sums cancel)."""

    def __init__(self, eps, n_mu: int, n_e: int, species=(0, 1, 2), weights=None, sin2w: float = 0.23,
                 g2: float = 1.0, norm: float = 1.0, eta_fp64: float = 0.0, precision: str = "mixed",
                 graph: bool = False, autotune: bool = False, split: bool = False, precise: bool = False,
                 device=None):
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
            sin2w=sin2w, g2=g2, norm=norm, eta_fp64=eta_fp64, prec=prec,
            flags=(capi.VX_USE_GRAPH if graph else 0) | (capi.VX_AUTOTUNE if autotune else 0)
            | (capi.VX_QUAD_SPLIT if split else 0) | (capi.VX_PRECISE if precise else 0))
        with torch.cuda.device(self.device):
            self._h = capi.vx_rates_create(cfg)

    # ------------------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            capi.vx_rates_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def entries_per_zone(self) -> int:
        """Kernel entries per zone and l: N^2."""
        return capi.vx_rates_entries_per_zone(self._h)

    def _batch(self, state, J, H, ray_offsets, stream=None):
        Z = state.shape[0]
        for name, t, shape in (("state", state, (Z, 4)), ("J", J, (Z, self.S, self.N)), ("H", H, (Z, self.S, self.N))):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shape:
                raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape {shape}")
            if t.device != self.device:
                raise ValueError(f"{name} is on {t.device}, the handle on {self.device}")
        offs, nr = self._offsets(ray_offsets, Z, stream)
        b = capi.vx_batch(n_rays=nr, n_zones=Z, ray_offsets=None if offs is None else ctypes.cast(offs.data_ptr(), capi._ip),
                          state=state.data_ptr(), J=J.data_ptr(), H=H.data_ptr())
        b._keep = offs
        return b

    def _offsets(self, ray_offsets, Z, stream=None):
        """Ray offsets as a device int32 tensor (host offsets are checked here and copied) and the
        ray count; (None, 1) without offsets."""
        offs = None
        nr = 1
        if ray_offsets is not None:
            if torch.is_tensor(ray_offsets) and ray_offsets.is_cuda:
                # device offsets: the library checks the partition on the device (vx_rates_check)
                if ray_offsets.dtype != torch.int32 or not ray_offsets.is_contiguous() or ray_offsets.dim() != 1:
                    raise ValueError("ray_offsets must be a contiguous 1-D int32 tensor")
                offs = ray_offsets
            else:
                h = np.ascontiguousarray(ray_offsets.cpu().numpy() if torch.is_tensor(ray_offsets) else ray_offsets,
                                         dtype=np.int64)
                if h.ndim != 1 or len(h) < 2 or h[0] != 0 or np.any(np.diff(h) < 0) or h[-1] != Z:
                    raise ValueError(f"ray_offsets must start at 0, not decrease and end at {Z}")
                offs = torch.from_numpy(h.astype(np.int32)).to(self.device, non_blocking=False)
                if stream is not None:
                    offs.record_stream(stream)
            nr = offs.shape[0] - 1
        return offs, nr

    def _check_out(self, name, t, shape, host=False):
        """Caller-supplied output (or seed) tensor: float64, contiguous, the given shape, on the
        handle's device (host=True: in host memory)."""
        ok = (torch.is_tensor(t) and t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == tuple(shape)
              and ((not t.is_cuda) if host else (t.is_cuda and t.device == self.device)))
        if not ok:
            where = "host" if host else f"{self.device}"
            raise ValueError(f"{name} must be a contiguous float64 tensor of shape {tuple(shape)} on {where}")

    def _alloc(self, Z):
        return {k: torch.empty((Z, self.S, self.N), dtype=torch.float64, device=self.device) for k in _OUT_KEYS}

    @staticmethod
    def _stream(stream):
        s = stream if stream is not None else torch.cuda.current_stream()
        return s.cuda_stream

    def evaluate(self, state, J, H, ray_offsets=None, phi: bool = False, out=None, stream=None) -> dict:
        """Rates j0, chi0, j1, chi1 of every zone ([Z][S][N] float64); phi=True adds the raw kernel
        of term I, [Z][2 dir][2 l][N][N]."""
        Z = state.shape[0]
        b = self._batch(state, J, H, ray_offsets, stream)
        if out is not None:
            for k in _OUT_KEYS:
                self._check_out(f"out[{k!r}]", out.get(k), (Z, self.S, self.N))
            if phi and "phi" in out:
                self._check_out("out['phi']", out["phi"], (Z, 2, 2, self.N, self.N))
        res = out if out is not None else self._alloc(Z)
        if phi and "phi" not in res:
            res["phi"] = torch.empty((Z, 2, 2, self.N, self.N), dtype=torch.float64, device=self.device)
        o = capi.vx_out(*(_ptr(res[k]) for k in _OUT_KEYS), _ptr(res.get("phi")) if phi else None)
        capi.vx_rates_eval(self._h, b, o, self._stream(stream))
        return res

    def adjoint(self, state, J, H, grad_out=None, jacobian: bool = True, forward: bool = False,
                ray_offsets=None, stream=None) -> dict:
        """One pass giving the Jacobian [Z][S][N][4][3] (d(j0,chi0,j1,chi1)/d(T,eta_e,Y_e)), the
        vector-Jacobian product grad_state [Z][4] for grad_out (dict of [Z][S][N] tensors) and/or
        the forward rates."""
        Z = state.shape[0]
        b = self._batch(state, J, H, ray_offsets, stream)
        self._check_seeds(grad_out, Z)
        res = {}
        if jacobian:
            res["jac"] = torch.empty((Z, self.S, self.N, 4, 3), dtype=torch.float64, device=self.device)
        g = None
        if grad_out is not None:
            g = capi.vx_out(*(_ptr(grad_out.get(k)) for k in _OUT_KEYS), None)
            res["grad_state"] = torch.empty((Z, 4), dtype=torch.float64, device=self.device)
        fwd = None
        if forward:
            res.update(self._alloc(Z))
            fwd = capi.vx_out(*(_ptr(res[k]) for k in _OUT_KEYS), None)
        capi.vx_rates_adjoint(self._h, b, g, _ptr(res.get("jac")), _ptr(res.get("grad_state")), fwd,
                              self._stream(stream))
        return res

    def spectral(self, state, J, H, grad_out=None, blocks: bool = True, forward: bool = False,
                 ray_offsets=None, stream=None) -> dict:
        """Derivatives with respect to the partner spectra from one forward pass: blocks
        [Z][S][4][N][N] (d j0/dJ, d chi0/dJ, d j1/dH, d chi1/dH of the spectrum each species reads)
        and/or, for grad_out (dict of [Z][S][N] tensors), grad_J and grad_H [Z][S][N] indexed by
        spectrum; forward=True adds the rates."""
        Z = state.shape[0]
        b = self._batch(state, J, H, ray_offsets, stream)
        self._check_seeds(grad_out, Z)
        res = {}
        if blocks:
            res["blocks"] = torch.empty((Z, self.S, 4, self.N, self.N), dtype=torch.float64, device=self.device)
        g = None
        if grad_out is not None:
            g = capi.vx_out(*(_ptr(grad_out.get(k)) for k in _OUT_KEYS), None)
            res["grad_J"] = torch.empty((Z, self.S, self.N), dtype=torch.float64, device=self.device)
            res["grad_H"] = torch.empty((Z, self.S, self.N), dtype=torch.float64, device=self.device)
        fwd = None
        if forward:
            res.update(self._alloc(Z))
            fwd = capi.vx_out(*(_ptr(res[k]) for k in _OUT_KEYS), None)
        capi.vx_rates_spectral(self._h, b, g, _ptr(res.get("grad_J")), _ptr(res.get("grad_H")), _ptr(res.get("blocks")),
                               fwd, self._stream(stream))
        return res

    def _check_seeds(self, grad_out, Z, host=False):
        if grad_out is None:
            return
        for k, v in grad_out.items():
            if k not in _OUT_KEYS:
                raise ValueError(f"grad_out has an unknown key {k!r}")
            if v is not None:
                self._check_out(f"grad_out[{k!r}]", v, (Z, self.S, self.N), host=host)

    def jacobian(self, state, J, H, **kw):
        return self.adjoint(state, J, H, jacobian=True, **kw)["jac"]

    def check(self, stream=None) -> bool:
        """Synchronise and read the device numeric flag: True if clean."""
        return capi.vx_rates_check(self._h, self._stream(stream)) == capi.VX_OK

    # ------------------------------------------------------------------------------------------
    def _host_batch(self, state, J, H, ray_offsets):
        arrs = [np.ascontiguousarray(torch.as_tensor(x).numpy() if torch.is_tensor(x) else x, dtype=np.float64)
                for x in (state, J, H)]
        Z = arrs[0].shape[0]
        for name, a, shape in zip(("state", "J", "H"), arrs, ((Z, 4), (Z, self.S, self.N), (Z, self.S, self.N))):
            if a.shape != shape:
                raise ValueError(f"{name} must have shape {shape}")
        offs = None if ray_offsets is None else np.ascontiguousarray(ray_offsets, dtype=np.int32)
        b = capi.vx_batch(n_rays=1 if offs is None else len(offs) - 1, n_zones=Z,
                          ray_offsets=None if offs is None else offs.ctypes.data_as(capi._ip),
                          state=arrs[0].ctypes.data, J=arrs[1].ctypes.data, H=arrs[2].ctypes.data)
        b._keep = (arrs, offs)
        return b, Z

    def _host_out(self, Z, out):
        if out is not None:
            for k in _OUT_KEYS:
                self._check_out(f"out[{k!r}]", out.get(k), (Z, self.S, self.N), host=True)
        res = out if out is not None else {k: torch.empty((Z, self.S, self.N), dtype=torch.float64, pin_memory=True)
                                           for k in _OUT_KEYS}
        return res, capi.vx_out(*(res[k].data_ptr() for k in _OUT_KEYS), None)

    def evaluate_host(self, state, J, H, ray_offsets=None, out=None) -> dict:
        """End-to-end call on host arrays (numpy or pinned torch CPU tensors): vx_rates_eval_host
        copies chunks of zones in, evaluates and copies the rates back, overlapping the copies of
        one chunk with the kernel of the next. Returns host tensors (pinned unless `out` given)."""
        b, Z = self._host_batch(state, J, H, ray_offsets)
        res, o = self._host_out(Z, out)
        with torch.cuda.device(self.device):
            capi.vx_rates_eval_host(self._h, b, o)
        return res

    def adjoint_host(self, state, J, H, forward: bool = True, ray_offsets=None, out=None, jac=None) -> dict:
        """End-to-end forward rates and Jacobian on host arrays (vx_rates_adjoint_host)."""
        b, Z = self._host_batch(state, J, H, ray_offsets)
        res, o = self._host_out(Z, out) if forward else ({}, None)
        if jac is not None:
            self._check_out("jac", jac, (Z, self.S, self.N, 4, 3), host=True)
        res["jac"] = jac if jac is not None else torch.empty((Z, self.S, self.N, 4, 3), dtype=torch.float64,
                                                             pin_memory=True)
        with torch.cuda.device(self.device):
            capi.vx_rates_adjoint_host(self._h, b, res["jac"].data_ptr(), o)
        return res


    def spectral_host(self, state, J, H, grad_out=None, blocks: bool = True, forward: bool = False,
                      ray_offsets=None) -> dict:
        """Spectral derivatives on host arrays (vx_rates_spectral_host): blocks and/or, for host
        seeds grad_out, grad_J and grad_H; forward=True adds the rates."""
        b, Z = self._host_batch(state, J, H, ray_offsets)
        res = {}
        pin = dict(dtype=torch.float64, pin_memory=True)
        if blocks:
            res["blocks"] = torch.empty((Z, self.S, 4, self.N, self.N), **pin)
        g = None
        if grad_out is not None:
            seeds = {k: np.ascontiguousarray(torch.as_tensor(v).numpy() if torch.is_tensor(v) else v, dtype=np.float64)
                     for k, v in grad_out.items() if v is not None}
            g = capi.vx_out(*((seeds[k].ctypes.data if k in seeds else None) for k in _OUT_KEYS), None)
            g._keep = seeds
            res["grad_J"] = torch.empty((Z, self.S, self.N), **pin)
            res["grad_H"] = torch.empty((Z, self.S, self.N), **pin)
        fwd = None
        if forward:
            fw, fwd = self._host_out(Z, None)
            res.update(fw)
        with torch.cuda.device(self.device):
            capi.vx_rates_spectral_host(self._h, b, g, _ptr(res.get("grad_J")), _ptr(res.get("grad_H")),
                                        _ptr(res.get("blocks")), fwd)
        return res


class VxRatesFn(torch.autograd.Function):
    """(j0, chi0, j1, chi1) = f(state, J, H): forward through vx_rates_eval; backward through the
    adjoint kernel (state: T, eta_e; the Y_e and rho entries are zero for this process) and the
    spectral kernel (J, H), each in vector-Jacobian mode and only for the inputs that need it."""

    @staticmethod
    def forward(ctx, rates: PairRates, state, J, H):
        out = rates.evaluate(state, J, H)
        ctx.rates = rates
        ctx.save_for_backward(state, J, H)
        return tuple(out[k] for k in _OUT_KEYS)

    @staticmethod
    def backward(ctx, *grads):
        state, J, H = ctx.saved_tensors
        g = {k: (gr.contiguous() if gr is not None else None) for k, gr in zip(_OUT_KEYS, grads)}
        gs = gJ = gH = None
        if ctx.needs_input_grad[1]:
            gs = ctx.rates.adjoint(state, J, H, grad_out=g, jacobian=False)["grad_state"]
        if ctx.needs_input_grad[2] or ctx.needs_input_grad[3]:
            res = ctx.rates.spectral(state, J, H, grad_out=g, blocks=False)
            gJ = res["grad_J"] if ctx.needs_input_grad[2] else None
            gH = res["grad_H"] if ctx.needs_input_grad[3] else None
        return None, gs, gJ, gH
