"""Seeded synthetic inputs for the e+e- pair-process rate kernel.

This module is shared by the CPU oracle and the GPU path. It holds no arithmetic of the
rate kernel itself: it only draws zone states, energy-bin centres and partner neutrino
spectra, the way a hydrodynamics/transport code would hand them to the rate module.

The paper's progenitor models are not available, so every workload is synthetic. The
shapes follow the paper's setting: rays of radial zones (ray-by-ray transport, paper
sec. 2.1-2.2), a logarithmic neutrino-energy grid, and Fermi-Dirac-like neutrino spectra
whose angular moments J (0th) and H (1st) are the occupation moments of the paper's
moment equation (sec. 2.1).

Workloads (seed 0 unless given):
  1  one ray x 64 zones, 17 bins 1-300 MeV, 16x32 quadrature, independent draws per zone
  2  one ray x 400 zones, 21 bins 1-380 MeV, 32x64, radial profiles with 5 % noise
  3  2048 rays of 300..550 zones, 21 bins, 32x64, profiles as 2
  4  4096 rays x 400 zones, 21 bins, 32x64, profiles as 2
  5  16200 rays x 400 zones, 21 bins, 16x48, profiles as 2 with eta_e stretched to 0-60

Every ray draws from its own counter-derived stream SeedSequence([seed, workload, ray]),
so any subset of rays is reproduced exactly without generating the rest.
"""
from __future__ import annotations

import numpy as np

NU_E, NU_EBAR, NU_X = 0, 1, 2

WORKLOADS = {
    1: dict(name="1ray-64z-17b-16x32", n_rays=1, ray_len=(64, 64), n_bins=17, e_min=1.0,
            e_max=300.0, n_mu=16, n_e=32, profile=None, eta_max=20.0),
    2: dict(name="1ray-400z-21b-32x64", n_rays=1, ray_len=(400, 400), n_bins=21, e_min=1.0,
            e_max=380.0, n_mu=32, n_e=64, profile="radial", eta_max=20.0),
    3: dict(name="2048ray-300to550z-21b-32x64", n_rays=2048, ray_len=(300, 550), n_bins=21,
            e_min=1.0, e_max=380.0, n_mu=32, n_e=64, profile="radial", eta_max=20.0),
    4: dict(name="4096ray-400z-21b-32x64", n_rays=4096, ray_len=(400, 400), n_bins=21,
            e_min=1.0, e_max=380.0, n_mu=32, n_e=64, profile="radial", eta_max=20.0),
    5: dict(name="16200ray-400z-21b-16x48-eta60", n_rays=16200, ray_len=(400, 400), n_bins=21,
            e_min=1.0, e_max=380.0, n_mu=16, n_e=48, profile="radial", eta_max=60.0),
}

SPECIES = (NU_E, NU_EBAR, NU_X)


def energy_centres(n_bins: int, e_min: float, e_max: float) -> np.ndarray:
    """Logarithmically spaced bin centres e_min * (e_max/e_min)**(i/(n-1)), MeV."""
    i = np.arange(n_bins, dtype=np.float64)
    return e_min * (e_max / e_min) ** (i / (n_bins - 1))


def ray_lengths(workload: int, seed: int = 0) -> np.ndarray:
    w = WORKLOADS[workload]
    lo, hi = w["ray_len"]
    if lo == hi:
        return np.full(w["n_rays"], lo, dtype=np.int64)
    rng = np.random.default_rng(np.random.SeedSequence([seed, workload, 0x7A7]))
    return rng.integers(lo, hi + 1, size=w["n_rays"]).astype(np.int64)


def _ray(workload: int, seed: int, ray: int, n_zones: int, eps: np.ndarray, n_species: int):
    w = WORKLOADS[workload]
    rng = np.random.default_rng(np.random.SeedSequence([seed, workload, ray]))
    if w["profile"] is None:
        T = np.exp(rng.uniform(np.log(1.0), np.log(30.0), n_zones))
        eta = rng.uniform(0.0, w["eta_max"], n_zones)
        ye = rng.uniform(0.1, 0.5, n_zones)
        rho = np.exp(rng.uniform(np.log(1e9), np.log(1e14), n_zones))
        flux = rng.uniform(0.0, 0.5, n_zones)
    else:
        x = np.arange(n_zones, dtype=np.float64) / max(n_zones - 1, 1)
        noise = 1.0 + 0.05 * rng.uniform(-1.0, 1.0, (4, n_zones))
        T = 30.0 * (1.0 / 30.0) ** x * noise[0]
        eta = np.maximum(w["eta_max"] * (1.0 - x) * noise[1], 0.0)
        rho = 10.0 ** (14.0 - 5.0 * x) * noise[2]
        ye = (0.3 + 0.2 * x) * noise[3]
        flux = 0.5 * x
    eta_nu = rng.uniform(0.0, 5.0, (n_zones, n_species))
    state = np.stack([T, eta, ye, rho], axis=1)
    # partner spectra: Fermi-Dirac occupation at the zone temperature, flux factor H/J
    arg = eps[None, None, :] / T[:, None, None] - eta_nu[:, :, None]
    J = 1.0 / (np.exp(np.minimum(arg, 700.0)) + 1.0)
    H = flux[:, None, None] * J
    return state, J, H


def make_batch(workload: int, seed: int = 0, rays=None, n_species: int = 3) -> dict:
    """Synthetic batch for a workload: bin centres, quadrature sizes, ray offsets, state, J, H.

    rays: None for all rays, else an iterable of ray indices (a seeded subset).
    state is [Z][4] float64 (T [MeV], eta_e, Y_e, rho [g/cm^3]); J, H are [Z][S][N] float64
    occupation moments of each species' own spectrum; species order nu_e, anti-nu_e, nu_x.
    """
    w = WORKLOADS[workload]
    eps = energy_centres(w["n_bins"], w["e_min"], w["e_max"])
    lens_all = ray_lengths(workload, seed)
    ray_ids = np.arange(w["n_rays"]) if rays is None else np.asarray(list(rays), dtype=np.int64)
    lens = lens_all[ray_ids]
    offsets = np.zeros(len(ray_ids) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lens)
    Z = int(offsets[-1])
    S = n_species
    state = np.empty((Z, 4))
    J = np.empty((Z, S, w["n_bins"]))
    H = np.empty((Z, S, w["n_bins"]))
    for k, r in enumerate(ray_ids):
        a, b = offsets[k], offsets[k + 1]
        state[a:b], J[a:b], H[a:b] = _ray(workload, seed, int(r), int(lens[k]), eps, S)
    return dict(workload=workload, name=w["name"], eps=eps, n_mu=w["n_mu"], n_e=w["n_e"],
                species=np.array(SPECIES[:S], dtype=np.int32), ray_offsets=offsets.astype(np.int32),
                state=state, J=J, H=H, rays=ray_ids)


def random_zones(n_zones: int, seed: int, T_range=(1.0, 30.0), eta_range=(0.0, 20.0),
                 n_bins: int = 17, n_species: int = 3):
    """Independent zone draws (log-uniform T, uniform eta) for small parity and edge cases."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xE5]))
    T = np.exp(rng.uniform(np.log(T_range[0]), np.log(T_range[1]), n_zones))
    eta = rng.uniform(eta_range[0], eta_range[1], n_zones)
    ye = rng.uniform(0.1, 0.5, n_zones)
    rho = np.exp(rng.uniform(np.log(1e9), np.log(1e14), n_zones))
    J = rng.uniform(0.0, 1.0, (n_zones, n_species, n_bins))
    H = rng.uniform(0.0, 0.5, (n_zones, n_species, n_bins)) * J
    return np.stack([T, eta, ye, rho], axis=1), J, H
