"""Seeded synthetic per-ray Newton systems (block tridiagonal) for the batched solve.

Shared by the oracle and the GPU path; it only draws and places numbers (no arithmetic of the
solve). No progenitor models exist here, so the systems are synthetic, shaped like the Jacobian of
one implicit radial step of a two-moment neutrino scheme (paper sec. 2.1-2.2):

* Unknowns per zone: the moments J and H of the two species the pair process couples (nu_e and its
  partner nu_ebar), N energy bins each: m = 4N, ordered [species][moment][bin]. (A nu_x system,
  whose partner is itself, has m = 2N: ``pair=False``.)
* Diagonal block B_k = I + D_k - P_k: D_k is the diagonal of absorption-like opacities times the
  time step (log-uniform over six decades, rising towards the centre of the ray); P_k couples each
  species' J to its partner's J over all bins, and H to H, with non-negative entries whose row sum
  is rho_k times that row's opacity (rho_k uniform in [0.1, 0.9]), the structure of the pair
  process's d(source)/d(J, H) blocks.
* Off-diagonal blocks: the radial flux terms couple J of zone k to H of zones k -/+ 1 and H to J,
  bin by bin: A_k = -c_k X, C_k = +c_k X with X the J <-> H exchange of each (species, bin), the H
  rows weighted by an Eddington factor in [1/3, 1], and c_k log-uniform in [0.01, 3].
* Right-hand sides are standard normal.

Every ray draws from SeedSequence([seed, 0xB7D, ray]), so any subset of rays is reproduced exactly.
"""
from __future__ import annotations

import numpy as np


def _ray_newton(seed: int, ray: int, n: int, N: int, pair: bool):
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xB7D, ray]))
    S = 2 if pair else 1
    m = 2 * S * N
    x = np.arange(n) / max(n - 1, 1)
    # opacity x time step per (zone, species, moment, bin): centre of the ray optically thick
    kap = 10.0 ** (3.0 - 6.0 * x[:, None, None, None] + rng.uniform(-0.5, 0.5, (n, S, 2, N)))
    rho = rng.uniform(0.1, 0.9, n)
    c = 10.0 ** rng.uniform(-2.0, np.log10(3.0), n)
    fedd = rng.uniform(1.0 / 3.0, 1.0, (n, S, N))
    w = rng.uniform(0.0, 1.0, (n, S, 2, N, N))  # pair coupling of (species, moment) rows to the partner
    w *= (rho[:, None, None, None] * kap)[..., None] / w.sum(axis=-1, keepdims=True)
    d = rng.standard_normal((n, m))
    A = np.zeros((n, m, m))
    B = np.zeros((n, m, m))
    C = np.zeros((n, m, m))
    diag = np.arange(m)
    B[:, diag, diag] = 1.0 + kap.reshape(n, m)
    ii = np.arange(N)
    for s in range(S):
        sp = (1 - s) if pair else s  # partner species
        for q in range(2):
            r0, c0 = (2 * s + q) * N, (2 * sp + q) * N
            B[:, r0:r0 + N, c0:c0 + N] -= w[:, s, q]
        # flux coupling: J_s(i) <- H_s(i) of the neighbours, H_s(i) <- J_s(i)
        rJ, rH = 2 * s * N + ii, (2 * s + 1) * N + ii
        A[1:, rJ, rH] = -c[1:, None]
        A[1:, rH, rJ] = -(c[:, None] * fedd[:, s])[1:]
        C[:-1, rJ, rH] = c[:-1, None]
        C[:-1, rH, rJ] = (c[:, None] * fedd[:, s])[:-1]
    return A, B, C, d


def newton_system(lengths, n_bins: int = 21, pair: bool = True, seed: int = 0, rays=None) -> dict:
    """Rays of the given zone counts (or the listed subset of them): blocks A, B, C [Z][m][m],
    right-hand side d [Z][m] and offsets [n_rays + 1] (int32)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    sel = range(len(lengths)) if rays is None else list(rays)
    parts = [_ray_newton(seed, r, int(lengths[r]), n_bins, pair) for r in sel]
    m = 4 * n_bins if pair else 2 * n_bins
    offsets = np.zeros(len(parts) + 1, np.int32)
    offsets[1:] = np.cumsum([p[0].shape[0] for p in parts])
    cat = [np.concatenate([p[i] for p in parts]) if parts else np.zeros((0, m, m) if i < 3 else (0, m))
           for i in range(4)]
    return dict(A=cat[0], B=cat[1], C=cat[2], d=cat[3], offsets=offsets, m=m)


def random_system(lengths, m: int, seed: int = 0, margin: float = 0.5) -> dict:
    """Generic dense blocks (uniform entries) with block rows made diagonally dominant by
    ``margin`` (the diagonal exceeds the row's other absolute entries, over all three blocks, by
    margin x that sum + 1)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xB7E, m]))
    Z = int(lengths.sum())
    A = rng.uniform(-1.0, 1.0, (Z, m, m))
    B = rng.uniform(-1.0, 1.0, (Z, m, m))
    C = rng.uniform(-1.0, 1.0, (Z, m, m))
    offsets = np.zeros(len(lengths) + 1, np.int32)
    offsets[1:] = np.cumsum(lengths)
    for r in range(len(lengths)):  # no coupling past the ends of a ray
        if lengths[r] > 0:
            A[offsets[r]] = 0.0
            C[offsets[r + 1] - 1] = 0.0
    diag = np.arange(m)
    off = np.abs(A).sum(2) + np.abs(C).sum(2) + np.abs(B).sum(2) - np.abs(B[:, diag, diag])
    sign = np.where(rng.uniform(size=(Z, m)) < 0.5, -1.0, 1.0)
    B[:, diag, diag] = sign * ((1.0 + margin) * off + 1.0)
    d = rng.standard_normal((Z, m))
    return dict(A=A, B=B, C=C, d=d, offsets=offsets, m=m)
