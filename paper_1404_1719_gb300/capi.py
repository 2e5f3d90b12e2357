"""ctypes binding of the C ABI in include/vx_rates.h and include/vx_btd.h: same names, argument
marshalling only.

The shared library is built in-tree by ``paper_1404_1719_gb300._build.build()``. There is no
fallback: if it is missing or cannot be loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

VX_OK, VX_ERR_INVALID_ARG, VX_ERR_CUDA, VX_ERR_OOM, VX_ERR_NUMERIC, VX_ERR_UNSUPPORTED, VX_ERR_TIMEOUT = range(7)
VX_PREC_FP64, VX_PREC_MIXED = 0, 1
VX_NU_E, VX_NU_EBAR, VX_NU_X = 0, 1, 2
VX_USE_GRAPH, VX_AUTOTUNE, VX_QUAD_SPLIT, VX_PRECISE = 1, 2, 4, 8

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class vx_config(ctypes.Structure):
    _fields_ = [("n_bins", ctypes.c_int), ("eps", _dp), ("weights", _dp), ("n_mu", ctypes.c_int),
                ("n_e", ctypes.c_int), ("n_species", ctypes.c_int), ("species", _ip),
                ("sin2w", ctypes.c_double), ("g2", ctypes.c_double), ("norm", ctypes.c_double),
                ("eta_fp64", ctypes.c_double), ("prec", ctypes.c_int), ("flags", ctypes.c_uint)]


class vx_batch(ctypes.Structure):
    _fields_ = [("n_rays", ctypes.c_int), ("n_zones", ctypes.c_longlong), ("ray_offsets", _ip),
                ("state", ctypes.c_void_p), ("J", ctypes.c_void_p), ("H", ctypes.c_void_p)]


class vx_out(ctypes.Structure):
    _fields_ = [("j0", ctypes.c_void_p), ("chi0", ctypes.c_void_p), ("j1", ctypes.c_void_p),
                ("chi1", ctypes.c_void_p), ("phi", ctypes.c_void_p)]


class vx_pipe_rates(ctypes.Structure):
    _fields_ = [("ffma", ctypes.c_double), ("ffma2", ctypes.c_double), ("dfma", ctypes.c_double),
                ("ex2", ctypes.c_double), ("rcp", ctypes.c_double), ("mma_tf32", ctypes.c_double),
                ("mma_bf16", ctypes.c_double), ("sm_mhz", ctypes.c_double), ("n_sm", ctypes.c_int)]


class VxError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {vx_status_string(status)}: {vx_last_error()}")


SYMBOLS = ("vx_rates_create", "vx_rates_eval", "vx_rates_adjoint", "vx_rates_check",
           "vx_rates_entries_per_zone", "vx_rates_destroy", "vx_status_string", "vx_last_error",
           "vx_rates_eval_noalloc", "vx_rates_spectral", "vx_rates_eval_host", "vx_rates_adjoint_host",
           "vx_rates_spectral_host", "vx_btd_create", "vx_btd_solve", "vx_btd_check", "vx_btd_destroy",
           "vx_probe_pipes", "vx_nes_create", "vx_nes_eval", "vx_nes_adjoint", "vx_nes_check", "vx_nes_destroy",
           "vx_eos_eta", "vx_eos_chain", "vx_nes_eval_host", "vx_nes_adjoint_host", "vx_abs_create", "vx_abs_eval", "vx_abs_adjoint", "vx_abs_check",
           "vx_abs_destroy")

_lib = None


def lib(path: str | None = None):
    """Load libvx_rates.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1404_1719_gb300._build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    L.vx_rates_create.argtypes = [ctypes.POINTER(vx_config), ctypes.POINTER(ctypes.c_void_p)]
    L.vx_rates_create.restype = ctypes.c_int
    L.vx_rates_eval.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.POINTER(vx_out), ctypes.c_void_p]
    L.vx_rates_eval.restype = ctypes.c_int
    L.vx_rates_adjoint.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.POINTER(vx_out), ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.POINTER(vx_out), ctypes.c_void_p]
    L.vx_rates_adjoint.restype = ctypes.c_int
    L.vx_rates_spectral.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.POINTER(vx_out), ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(vx_out), ctypes.c_void_p]
    L.vx_rates_spectral.restype = ctypes.c_int
    L.vx_rates_eval_host.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.POINTER(vx_out)]
    L.vx_rates_eval_host.restype = ctypes.c_int
    L.vx_rates_adjoint_host.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.c_void_p,
                                        ctypes.POINTER(vx_out)]
    L.vx_rates_adjoint_host.restype = ctypes.c_int
    L.vx_rates_spectral_host.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.POINTER(vx_out),
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(vx_out)]
    L.vx_rates_spectral_host.restype = ctypes.c_int
    L.vx_rates_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.vx_rates_check.restype = ctypes.c_int
    L.vx_rates_entries_per_zone.argtypes = [ctypes.c_void_p]
    L.vx_rates_entries_per_zone.restype = ctypes.c_longlong
    L.vx_rates_destroy.argtypes = [ctypes.c_void_p]
    L.vx_rates_destroy.restype = None
    L.vx_status_string.argtypes = [ctypes.c_int]
    L.vx_status_string.restype = ctypes.c_char_p
    L.vx_rates_eval_noalloc.argtypes = [ctypes.POINTER(vx_config), ctypes.POINTER(vx_batch), ctypes.POINTER(vx_out),
                                        ctypes.c_void_p]
    L.vx_rates_eval_noalloc.restype = ctypes.c_int
    L.vx_last_error.argtypes = []
    L.vx_last_error.restype = ctypes.c_char_p
    L.vx_btd_create.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    L.vx_btd_create.restype = ctypes.c_int
    L.vx_btd_solve.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong] + [ctypes.c_void_p] * 7
    L.vx_btd_solve.restype = ctypes.c_int
    L.vx_btd_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.vx_btd_check.restype = ctypes.c_int
    L.vx_btd_destroy.argtypes = [ctypes.c_void_p]
    L.vx_btd_destroy.restype = None
    L.vx_probe_pipes.argtypes = [ctypes.POINTER(vx_pipe_rates), ctypes.c_void_p]
    L.vx_probe_pipes.restype = ctypes.c_int
    L.vx_nes_create.argtypes = [ctypes.POINTER(vx_config), ctypes.POINTER(ctypes.c_void_p)]
    L.vx_nes_create.restype = ctypes.c_int
    L.vx_nes_eval.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.POINTER(vx_out), ctypes.c_void_p]
    L.vx_nes_eval.restype = ctypes.c_int
    L.vx_nes_adjoint.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.c_void_p, ctypes.POINTER(vx_out),
                                 ctypes.c_void_p]
    L.vx_nes_adjoint.restype = ctypes.c_int
    L.vx_nes_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.vx_nes_check.restype = ctypes.c_int
    L.vx_nes_destroy.argtypes = [ctypes.c_void_p]
    L.vx_nes_destroy.restype = None
    L.vx_nes_eval_host.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.POINTER(vx_out)]
    L.vx_nes_eval_host.restype = ctypes.c_int
    L.vx_nes_adjoint_host.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.c_void_p,
                                      ctypes.POINTER(vx_out)]
    L.vx_nes_adjoint_host.restype = ctypes.c_int
    L.vx_abs_create.argtypes = [ctypes.POINTER(vx_config), ctypes.POINTER(ctypes.c_void_p)]
    L.vx_abs_create.restype = ctypes.c_int
    L.vx_abs_eval.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.POINTER(vx_out), ctypes.c_void_p]
    L.vx_abs_eval.restype = ctypes.c_int
    L.vx_abs_adjoint.argtypes = [ctypes.c_void_p, ctypes.POINTER(vx_batch), ctypes.c_void_p, ctypes.POINTER(vx_out),
                                 ctypes.c_void_p]
    L.vx_abs_adjoint.restype = ctypes.c_int
    L.vx_abs_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.vx_abs_check.restype = ctypes.c_int
    L.vx_abs_destroy.argtypes = [ctypes.c_void_p]
    L.vx_abs_destroy.restype = None
    L.vx_eos_eta.argtypes = [ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.vx_eos_eta.restype = ctypes.c_int
    L.vx_eos_chain.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]
    L.vx_eos_chain.restype = ctypes.c_int
    _lib = L
    return L


def vx_status_string(s: int) -> str:
    return lib().vx_status_string(int(s)).decode()


def vx_last_error() -> str:
    return lib().vx_last_error().decode()


def _check(status: int, where: str):
    if status != VX_OK:
        raise VxError(status, where)


def vx_rates_create(cfg: vx_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().vx_rates_create(ctypes.byref(cfg), ctypes.byref(h)), "vx_rates_create")
    return h


def vx_rates_eval(h, batch: vx_batch, out: vx_out, stream: int = 0) -> None:
    _check(lib().vx_rates_eval(h, ctypes.byref(batch), ctypes.byref(out), ctypes.c_void_p(stream)), "vx_rates_eval")


def vx_rates_eval_noalloc(cfg: vx_config, batch: vx_batch, out: vx_out, stream: int = 0) -> None:
    """Forward rates without a handle and without any allocation by the library (see the header
    for its limits and the shared scratch it uses)."""
    _check(lib().vx_rates_eval_noalloc(ctypes.byref(cfg), ctypes.byref(batch), ctypes.byref(out),
                                       ctypes.c_void_p(stream)), "vx_rates_eval_noalloc")


def vx_rates_adjoint(h, batch: vx_batch, grad_out: vx_out | None, jac: int | None, grad_state: int | None,
                     fwd: vx_out | None, stream: int = 0) -> None:
    st = lib().vx_rates_adjoint(h, ctypes.byref(batch), ctypes.byref(grad_out) if grad_out is not None else None,
                                ctypes.c_void_p(jac or 0), ctypes.c_void_p(grad_state or 0),
                                ctypes.byref(fwd) if fwd is not None else None, ctypes.c_void_p(stream))
    _check(st, "vx_rates_adjoint")


def vx_rates_spectral(h, batch: vx_batch, grad_out: vx_out | None, grad_J: int | None, grad_H: int | None,
                      blocks: int | None, fwd: vx_out | None, stream: int = 0) -> None:
    st = lib().vx_rates_spectral(h, ctypes.byref(batch), ctypes.byref(grad_out) if grad_out is not None else None,
                                 ctypes.c_void_p(grad_J or 0), ctypes.c_void_p(grad_H or 0),
                                 ctypes.c_void_p(blocks or 0), ctypes.byref(fwd) if fwd is not None else None,
                                 ctypes.c_void_p(stream))
    _check(st, "vx_rates_spectral")


def vx_rates_eval_host(h, batch: vx_batch, out: vx_out) -> None:
    """Host arrays in and out (see the header); synchronous."""
    _check(lib().vx_rates_eval_host(h, ctypes.byref(batch), ctypes.byref(out)), "vx_rates_eval_host")


def vx_rates_adjoint_host(h, batch: vx_batch, jac: int | None, fwd: vx_out | None) -> None:
    """Host arrays in and out (see the header); synchronous."""
    _check(lib().vx_rates_adjoint_host(h, ctypes.byref(batch), ctypes.c_void_p(jac or 0),
                                       ctypes.byref(fwd) if fwd is not None else None), "vx_rates_adjoint_host")


def vx_rates_spectral_host(h, batch: vx_batch, grad_out: vx_out | None, grad_J: int | None, grad_H: int | None,
                           blocks: int | None, fwd: vx_out | None) -> None:
    """Host arrays in and out (see the header); synchronous."""
    st = lib().vx_rates_spectral_host(h, ctypes.byref(batch), ctypes.byref(grad_out) if grad_out is not None else None,
                                      ctypes.c_void_p(grad_J or 0), ctypes.c_void_p(grad_H or 0),
                                      ctypes.c_void_p(blocks or 0), ctypes.byref(fwd) if fwd is not None else None)
    _check(st, "vx_rates_spectral_host")


def vx_rates_check(h, stream: int = 0) -> int:
    """Returns the status (VX_OK or VX_ERR_NUMERIC) instead of raising on a numeric flag."""
    st = lib().vx_rates_check(h, ctypes.c_void_p(stream))
    if st not in (VX_OK, VX_ERR_NUMERIC):
        raise VxError(st, "vx_rates_check")
    return st


def vx_rates_entries_per_zone(h) -> int:
    return int(lib().vx_rates_entries_per_zone(h))


def vx_rates_destroy(h) -> None:
    lib().vx_rates_destroy(h)


VX_BTD_MAX_M, VX_BTD_MAX_REFINE = 128, 8


def vx_btd_create(m: int, max_zones: int, n_refine: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().vx_btd_create(int(m), int(max_zones), int(n_refine), ctypes.byref(h)), "vx_btd_create")
    return h


def vx_btd_solve(h, n_rays: int, n_zones: int, ray_offsets: int, A: int, B: int, C: int, d: int, x: int,
                 stream: int = 0) -> None:
    st = lib().vx_btd_solve(h, int(n_rays), int(n_zones), *(ctypes.c_void_p(p or 0) for p in (ray_offsets, A, B, C, d, x)),
                            ctypes.c_void_p(stream))
    _check(st, "vx_btd_solve")


def vx_btd_check(h, stream: int = 0) -> int:
    """VX_OK or VX_ERR_NUMERIC (other failures raise)."""
    st = lib().vx_btd_check(h, ctypes.c_void_p(stream))
    if st not in (VX_OK, VX_ERR_NUMERIC):
        raise VxError(st, "vx_btd_check")
    return st


def vx_btd_destroy(h) -> None:
    lib().vx_btd_destroy(h)


def vx_probe_pipes(stream: int = 0) -> dict:
    """Measured pipe rates of the current device (per SM per clock; include/vx_probe.h)."""
    r = vx_pipe_rates()
    _check(lib().vx_probe_pipes(ctypes.byref(r), ctypes.c_void_p(stream)), "vx_probe_pipes")
    return {k: getattr(r, k) for k, _ in vx_pipe_rates._fields_}


def vx_nes_create(cfg: vx_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().vx_nes_create(ctypes.byref(cfg), ctypes.byref(h)), "vx_nes_create")
    return h


def vx_nes_eval(h, batch: vx_batch, out: vx_out, stream: int = 0) -> None:
    _check(lib().vx_nes_eval(h, ctypes.byref(batch), ctypes.byref(out), ctypes.c_void_p(stream)), "vx_nes_eval")


def vx_nes_adjoint(h, batch: vx_batch, jac: int, fwd: vx_out | None, stream: int = 0) -> None:
    _check(lib().vx_nes_adjoint(h, ctypes.byref(batch), ctypes.c_void_p(jac or 0),
                                ctypes.byref(fwd) if fwd is not None else None, ctypes.c_void_p(stream)),
           "vx_nes_adjoint")


def vx_nes_check(h, stream: int = 0) -> int:
    """VX_OK or VX_ERR_NUMERIC (other failures raise)."""
    st = lib().vx_nes_check(h, ctypes.c_void_p(stream))
    if st not in (VX_OK, VX_ERR_NUMERIC):
        raise VxError(st, "vx_nes_check")
    return st


def vx_nes_destroy(h) -> None:
    lib().vx_nes_destroy(h)


def vx_nes_eval_host(h, batch: vx_batch, out: vx_out) -> None:
    """Host arrays in and out (see the header); synchronous."""
    _check(lib().vx_nes_eval_host(h, ctypes.byref(batch), ctypes.byref(out)), "vx_nes_eval_host")


def vx_nes_adjoint_host(h, batch: vx_batch, jac: int, fwd: vx_out | None) -> None:
    """Host arrays in and out (see the header); synchronous."""
    _check(lib().vx_nes_adjoint_host(h, ctypes.byref(batch), ctypes.c_void_p(jac or 0),
                                     ctypes.byref(fwd) if fwd is not None else None), "vx_nes_adjoint_host")


def vx_abs_create(cfg: vx_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().vx_abs_create(ctypes.byref(cfg), ctypes.byref(h)), "vx_abs_create")
    return h


def vx_abs_eval(h, batch: vx_batch, out: vx_out, stream: int = 0) -> None:
    _check(lib().vx_abs_eval(h, ctypes.byref(batch), ctypes.byref(out), ctypes.c_void_p(stream)), "vx_abs_eval")


def vx_abs_adjoint(h, batch: vx_batch, jac: int | None, fwd: vx_out | None, stream: int = 0) -> None:
    _check(lib().vx_abs_adjoint(h, ctypes.byref(batch), ctypes.c_void_p(jac or 0),
                                ctypes.byref(fwd) if fwd is not None else None, ctypes.c_void_p(stream)),
           "vx_abs_adjoint")


def vx_abs_check(h, stream: int = 0) -> int:
    """VX_OK or VX_ERR_NUMERIC (other failures raise)."""
    st = lib().vx_abs_check(h, ctypes.c_void_p(stream))
    if st not in (VX_OK, VX_ERR_NUMERIC):
        raise VxError(st, "vx_abs_check")
    return st


def vx_abs_destroy(h) -> None:
    lib().vx_abs_destroy(h)


def vx_eos_eta(n_zones: int, state: int, deta: int | None, stream: int = 0) -> None:
    _check(lib().vx_eos_eta(int(n_zones), ctypes.c_void_p(state or 0), ctypes.c_void_p(deta or 0),
                            ctypes.c_void_p(stream)), "vx_eos_eta")


def vx_eos_chain(n_zones: int, rows: int, deta: int, jac_in: int, jac_out: int, stream: int = 0) -> None:
    _check(lib().vx_eos_chain(int(n_zones), int(rows), ctypes.c_void_p(deta or 0), ctypes.c_void_p(jac_in or 0),
                              ctypes.c_void_p(jac_out or 0), ctypes.c_void_p(stream)), "vx_eos_chain")
