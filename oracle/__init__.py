"""FP64 CPU oracle for the e+e- pair-process rate kernel -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. The product library never calls it, and it shares no code with the GPU path:
the arithmetic lives in ``vx_oracle.c`` (plain C, FP64, OpenMP over zones, no FMA contraction),
built by :func:`build` with gcc. This module only marshals numpy arrays through ctypes.

The kernel definition, the discrete rule and every reading of the paper the oracle adopts are
stated in the header comment of ``vx_oracle.c``.
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vx_oracle.c")
_SRC_NES = os.path.join(_HERE, "vx_nes_oracle.c")
_SRC_ABS = os.path.join(_HERE, "vx_abs_oracle.c")
_SO = os.path.join(_HERE, "libvx_oracle.so")
_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile vx_oracle.c, vx_nes_oracle.c and vx_abs_oracle.c into libvx_oracle.so (gcc, -O2,
    OpenMP when available)."""
    srcs = (_SRC, _SRC_NES, _SRC_ABS)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(os.path.getmtime(f) for f in srcs):
        return _SO
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
            "-o", _SO + ".tmp", *srcs, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)  # serial build without OpenMP
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.vxo_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
        lib.vxo_energy_weights.argtypes = [ctypes.c_int, _dp, _dp]
        lib.vxo_kernel_point.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.c_int, _dp, _dp,
                                                                 _dp, _dp, _dp]
        lib.vxo_kernel_point.restype = None
        lib.vxo_kernel_point_split.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.c_int, _dp, _dp,
                                                                       ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        lib.vxo_kernel_point_split.restype = None
        lib.vxo_phi_zone.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp]
        lib.vxo_phi_zone.restype = None
        lib.vxo_eval.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                 _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                 ctypes.c_int, ctypes.c_double, ctypes.c_int]
        lib.vxo_eval.restype = ctypes.c_int
        lib.vxo_gauss_laguerre.argtypes = [ctypes.c_int, _dp, _dp]
        lib.vxo_nes_nodes.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.vxo_nes_nodes.restype = None
        lib.vxo_nes_point.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp,
                                                              _dp, _dp, _dp]
        lib.vxo_nes_point.restype = None
        lib.vxo_nes_eval.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                     _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                     ctypes.c_int]
        lib.vxo_nes_eval.restype = ctypes.c_int
        lib.vxo_eos_eta.argtypes = [ctypes.c_long, _dp, _dp, _dp]
        lib.vxo_abs_eval.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _ip, ctypes.c_double, ctypes.c_longlong, _dp,
                                     _dp, _dp, _dp, _dp, _dp]
        lib.vxo_abs_eval.restype = None
        lib.vxo_eos_eta.restype = None
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def gauss_legendre(n: int):
    """Gauss-Legendre nodes (ascending) and weights on [-1, 1]."""
    x, w = np.empty(n), np.empty(n)
    if _load().vxo_gauss_legendre(n, _p(x), _p(w)) != 0:
        raise ValueError("bad node count")
    return x, w


def energy_weights(eps) -> np.ndarray:
    """w_i = eps_i^2 d(eps_i) for bin centres eps (edges at geometric midpoints)."""
    eps = _f64(eps)
    w = np.empty_like(eps)
    if _load().vxo_energy_weights(len(eps), _p(eps), _p(w)) != 0:
        raise ValueError("need at least two bins")
    return w


def kernel_point(eps, epsp, y, T, eta, n_e, boltzmann=False, grad=False, split=False):
    """K^X_dir(eps, eps', y) with G2 = 1: array [dir][X] (dir 0 = production, 1 = annihilation;
    X 0 = I, 1 = II); with grad=True also dK [dir][X][(d/dT, d/deta)]. split=True evaluates the
    split rule (two n_e/2-node panels meeting at the Fermi edge when it lies inside (E-, E+))."""
    tE, wE = gauss_legendre(n_e)
    K = np.empty(4)
    dK = np.empty(8) if grad else None
    if split:
        if n_e % 2:
            raise ValueError("the split rule needs an even n_e")
        tH, wH = gauss_legendre(n_e // 2)
        _load().vxo_kernel_point_split(float(eps), float(epsp), float(y), float(T), float(eta), int(boltzmann),
                                       n_e, _p(tE), _p(wE), n_e // 2, _p(tH), _p(wH), _p(K), _p(dK), None)
    else:
        _load().vxo_kernel_point(float(eps), float(epsp), float(y), float(T), float(eta), int(boltzmann),
                                 n_e, _p(tE), _p(wE), _p(K), _p(dK), None)
    return (K.reshape(2, 2), dK.reshape(2, 2, 2)) if grad else K.reshape(2, 2)


def phi_zone(eps, n_mu, n_e, T, eta, g2=1.0, boltzmann=False, grad=False, mag=False, split=False,
             eta_split=20.0):
    """Phi^dir_{l,X}(i,j) of one zone: array [dir][X][l][i][j] (and [.., 2] gradients); mag=True
    returns instead the same sums with |P_l| (the magnitude bounding the l = 1 rounding)."""
    eps = _f64(eps)
    n = len(eps)
    tmu, wmu = gauss_legendre(n_mu)
    tE, wE = gauss_legendre(n_e)
    phi = np.empty(8 * n * n)
    dphi = np.empty(16 * n * n) if grad else None
    pabs = np.empty(8 * n * n) if mag else None
    _load().vxo_phi_zone(n, _p(eps), n_mu, _p(tmu), _p(wmu), n_e, _p(tE), _p(wE), float(g2), float(T),
                         float(eta), int(boltzmann), int(split), float(eta_split), _p(phi), _p(dphi), _p(pabs),
                         None)
    if mag:
        return pabs.reshape(2, 2, 2, n, n)
    phi = phi.reshape(2, 2, 2, n, n)
    return (phi, dphi.reshape(2, 2, 2, n, n, 2)) if grad else phi


def evaluate(eps, n_mu, n_e, species, state, J, H, weights=None, sin2w=0.23, g2=1.0, norm=1.0,
             phi=False, jac=False, spectral=False, mag=False, split=False, eta_split=20.0, threads=0) -> dict:
    """Rates j0, chi0, j1, chi1 [Z][S][N] for every zone; optionally the K^I dump
    phi [Z][dir][l][N][N], the Jacobian jac [Z][S][N][4 outputs][3 inputs T, eta, Y_e], the
    spectral blocks dsrc [Z][S][4][N][N] (d j0/dJ, d chi0/dJ, d j1/dH, d chi1/dH of the partner
    spectrum; see vxo_eval), and with mag=True the magnitudes j1_abs, chi1_abs (phi_abs, jac_abs,
    dsrc_abs with the corresponding option): the same sums with every term replaced by its
    absolute value, which bound the rounding of results whose terms change sign (the l = 1
    projections and the derivatives). split=True selects the split discrete rule (n_e even) in
    zones with |eta| > eta_split (20, the GPU's default precision switch)."""
    eps = _f64(eps)
    state = _f64(state)
    J, H = _f64(J), _f64(H)
    species = np.ascontiguousarray(species, dtype=np.int32)
    n, S, Z = len(eps), len(species), state.shape[0]
    if J.shape != (Z, S, n) or H.shape != (Z, S, n) or state.shape != (Z, 4):
        raise ValueError("shape mismatch")
    out = {k: np.empty((Z, S, n)) for k in ("j0", "chi0", "j1", "chi1")}
    out["phi"] = np.empty((Z, 2, 2, n, n)) if phi else None
    out["jac"] = np.empty((Z, S, n, 4, 3)) if jac else None
    for k in ("j1_abs", "chi1_abs"):
        out[k] = np.empty((Z, S, n)) if mag else None
    out["phi_abs"] = np.empty((Z, 2, 2, n, n)) if (mag and phi) else None
    out["jac_abs"] = np.empty((Z, S, n, 4, 3)) if (mag and jac) else None
    out["dsrc"] = np.empty((Z, S, 4, n, n)) if spectral else None
    out["dsrc_abs"] = np.empty((Z, S, 4, n, n)) if (mag and spectral) else None
    w = None if weights is None else _f64(weights)
    used = _load().vxo_eval(n, _p(eps), _p(w), n_mu, n_e, S, species.ctypes.data_as(_ip), sin2w, g2, norm,
                            Z, _p(state), _p(J), _p(H), _p(out["j0"]), _p(out["chi0"]), _p(out["j1"]),
                            _p(out["chi1"]), _p(out["phi"]), _p(out["jac"]), _p(out["j1_abs"]),
                            _p(out["chi1_abs"]), _p(out["phi_abs"]), _p(out["jac_abs"]), _p(out["dsrc"]),
                            _p(out["dsrc_abs"]), int(bool(split)), float(eta_split), int(threads))
    if used < 0:
        raise ValueError("oracle rejected the arguments")
    out["threads"] = used
    return out


def partner_indices(species) -> np.ndarray:
    """Index, in the species list, of each species' partner spectrum: nu_e <-> anti-nu_e, nu_x with
    itself (the pairing vx_oracle.c uses; -1 where the partner is absent)."""
    sp = [int(x) for x in species]
    want = {0: 1, 1: 0, 2: 2}
    return np.array([sp.index(want[x]) if want[x] in sp else -1 for x in sp], dtype=np.int64)


def spectral_vjp(dsrc, species, g_j0, g_chi0, g_j1, g_chi1):
    """Vector-Jacobian product of seeds g_* [Z][S][N] with the spectral blocks dsrc [Z][S][4][N][N]:
    grad_J, grad_H [Z][S][N], indexed by the spectrum (each species' rates read its partner's)."""
    Z, S, _, N, _ = dsrc.shape
    pk = partner_indices(species)
    gJ = np.zeros((Z, S, N))
    gH = np.zeros((Z, S, N))
    for s in range(S):
        gJ[:, pk[s], :] += np.einsum("zij,zi->zj", dsrc[:, s, 0], g_j0[:, s]) + \
            np.einsum("zij,zi->zj", dsrc[:, s, 1], g_chi0[:, s])
        gH[:, pk[s], :] += np.einsum("zij,zi->zj", dsrc[:, s, 2], g_j1[:, s]) + \
            np.einsum("zij,zi->zj", dsrc[:, s, 3], g_chi1[:, s])
    return gJ, gH


# ---- inelastic neutrino-electron scattering (vx_nes_oracle.c) --------------------------------

def gauss_laguerre(n: int):
    """Gauss-Laguerre nodes (ascending) and weights for the weight e^{-x} on [0, inf)."""
    x, w = np.empty(n), np.empty(n)
    if _load().vxo_gauss_laguerre(n, _p(x), _p(w)) != 0:
        raise ValueError("bad node count")
    return x, w


@functools.lru_cache(maxsize=None)
def _nes_rules(n_e):
    if n_e % 3:
        raise ValueError("n_e must be a multiple of 3 (three panels)")
    n_p = n_e // 3
    tg, wg = gauss_legendre(n_p)
    xl, wl = gauss_laguerre(n_p)
    return n_p, tg, wg, xl, wl


def nes_nodes(eps, epsp, y, T, eta, n_e):
    """Electron energies E and weights W (dE included) of the three-panel rule at one point."""
    n_p, tg, wg, xl, wl = _nes_rules(n_e)
    E, W = np.empty(3 * n_p), np.empty(3 * n_p)
    _load().vxo_nes_nodes(float(eps), float(epsp), float(y), float(T), float(eta), n_p, _p(tg), _p(wg), _p(xl),
                          _p(wl), _p(E), _p(W))
    return E, W


def nes_point(eps, epsp, y, T, eta, n_e, boltzmann=False, grad=False, mag=False):
    """NES kernel R^dir_X(eps, eps', y) with G2 = 1: array [dir][X] (dir 0 = in, 1 = out; X 0 = I,
    1 = II); grad=True adds dK [dir][X][(d/dT, d/deta)], mag=True the sums of |terms|."""
    n_p, tg, wg, xl, wl = _nes_rules(n_e)
    K, dK, Ka = np.empty(4), np.empty(8), np.empty(4)
    _load().vxo_nes_point(float(eps), float(epsp), float(y), float(T), float(eta), int(boltzmann), n_p, _p(tg),
                          _p(wg), _p(xl), _p(wl), _p(K), _p(dK) if grad else None, _p(Ka))
    out = [K.reshape(2, 2)]
    if grad:
        out.append(dK.reshape(2, 2, 2))
    if mag:
        out.append(Ka.reshape(2, 2))
    return out[0] if len(out) == 1 else tuple(out)


def nes_evaluate(eps, n_mu, n_e, species, state, J, H, weights=None, sin2w=0.23, g2=1.0, norm=1.0, phi=False,
                 jac=False, mag=False, threads=0) -> dict:
    """NES rates j0 (in-scattering, J), chi0 (out-scattering, 1 - J), j1, chi1 (H) [Z][S][N] of every
    zone, with the source df/dt = (1 - f)(j0 - mu j1) - f (chi0 + mu chi1); optionally the kernel dump
    phi [Z][2 X][2 dir][2 l][N][N] (dir 0 = in, 1 = out), the Jacobian jac [Z][S][N][4][3]
    (d/dT, d/deta, d/dY_e = 0) and, with mag=True, the sums of |terms| (j1_abs, chi1_abs, phi_abs,
    jac_abs)."""
    eps = _f64(eps)
    state = _f64(state)
    J, H = _f64(J), _f64(H)
    species = np.ascontiguousarray(species, dtype=np.int32)
    n, S, Z = len(eps), len(species), state.shape[0]
    if J.shape != (Z, S, n) or H.shape != (Z, S, n) or state.shape != (Z, 4):
        raise ValueError("shape mismatch")
    out = {k: np.empty((Z, S, n)) for k in ("j0", "chi0", "j1", "chi1")}
    out["phi"] = np.empty((Z, 2, 2, 2, n, n)) if phi else None
    out["jac"] = np.empty((Z, S, n, 4, 3)) if jac else None
    for k in ("j1_abs", "chi1_abs"):
        out[k] = np.empty((Z, S, n)) if mag else None
    out["phi_abs"] = np.empty((Z, 2, 2, 2, n, n)) if (mag and phi) else None
    out["jac_abs"] = np.empty((Z, S, n, 4, 3)) if (mag and jac) else None
    w = None if weights is None else _f64(weights)
    used = _load().vxo_nes_eval(n, _p(eps), _p(w), n_mu, n_e, S, species.ctypes.data_as(_ip), sin2w, g2, norm, Z,
                                _p(state), _p(J), _p(H), _p(out["j0"]), _p(out["chi0"]), _p(out["j1"]),
                                _p(out["chi1"]), _p(out["phi"]), _p(out["jac"]), _p(out["j1_abs"]),
                                _p(out["chi1_abs"]), _p(out["phi_abs"]), _p(out["jac_abs"]), int(threads))
    if used < 0:
        raise ValueError("oracle rejected the arguments")
    out["threads"] = used
    return out


def eos_eta(state):
    """eta_e of every zone from T, Y_e, rho (state [Z][4]) by the massless electron-gas closure, and
    d eta / d(T, Y_e, rho) [Z][3]."""
    state = _f64(state)
    Z = state.shape[0]
    eta, deta = np.empty(Z), np.empty((Z, 3))
    _load().vxo_eos_eta(Z, _p(state), _p(eta), _p(deta))
    return eta, deta


def abs_evaluate(eps, species, state, g2=1.0, jac=False):
    """Charged-current absorption and emission rates on free nucleons (vx_abs_oracle.c): j0, chi0,
    j1, chi1 [Z][S][N] and, with jac=True, the Jacobian [Z][S][N][4][3] (d/dT, d/deta_e, d/dY_e)."""
    eps = _f64(eps)
    species = np.ascontiguousarray(species, dtype=np.int32)
    state = _f64(state)
    Z, S, N = state.shape[0], len(species), len(eps)
    out = {k: np.empty((Z, S, N)) for k in ("j0", "chi0", "j1", "chi1")}
    jc = np.empty((Z, S, N, 4, 3)) if jac else None
    _load().vxo_abs_eval(N, _p(eps), S, species.ctypes.data_as(_ip), float(g2), Z, _p(state),
                         *(_p(out[k]) for k in ("j0", "chi0", "j1", "chi1")), _p(jc) if jac else None)
    if jac:
        out["jac"] = jc
    return out
