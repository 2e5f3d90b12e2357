"""FP64 CPU oracle for the per-ray block-tridiagonal Newton solve -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import this
module; the product library never calls it and shares no code with it.

What is solved (paper sec. 2.1): the radial transport sweeps are implicit in time and run ray by
ray; each ray's time step is a non-linear system in the zone unknowns, solved by Newton-Raphson
iterations with an explicitly built Jacobian and a direct solve of the linearised system. A radial
difference scheme couples a zone only to its two neighbours, so that linear system is block
tridiagonal. For the zones k = 0 .. n-1 of one ray, with m unknowns per zone:

    A_k x_{k-1} + B_k x_k + C_k x_{k+1} = d_k,      (A_0 and C_{n-1} multiply nothing)

A, B, C are [Z][m][m] row-major blocks and d, x are [Z][m], concatenated over rays as
``offsets`` ([n_rays + 1], ray r owns zones offsets[r] .. offsets[r+1]-1).

The oracle solves each ray as the banded linear system it is, with no use of the block structure:
the ray's matrix goes into LAPACK band storage (2m - 1 sub- and super-diagonals) and
scipy.linalg.solve_banded factors it (LU with partial pivoting across the whole band). For tiny
systems :func:`solve_dense` writes out the full matrix and calls numpy.linalg.solve.
"""
from __future__ import annotations

import numpy as np


def dense_matrix(A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """The full (n m) x (n m) matrix of one ray from its blocks (each [n][m][m])."""
    n, m, _ = B.shape
    M = np.zeros((n * m, n * m))
    for k in range(n):
        r = slice(k * m, (k + 1) * m)
        M[r, r] = B[k]
        if k > 0:
            M[r, (k - 1) * m:k * m] = A[k]
        if k + 1 < n:
            M[r, (k + 1) * m:(k + 2) * m] = C[k]
    return M


def solve_dense(A, B, C, d) -> np.ndarray:
    """One ray by a dense solve (tiny systems only)."""
    n, m, _ = B.shape
    if n == 0:
        return np.zeros((0, m))
    return np.linalg.solve(dense_matrix(A, B, C), d.reshape(-1)).reshape(n, m)


def band_storage(A, B, C) -> tuple[np.ndarray, int]:
    """LAPACK band storage of one ray's matrix: ab[w + i - j, j] = M[i, j], w = 2m - 1 sub- and
    super-diagonals (a row of zone k reaches back to the first column of zone k - 1 and forward to
    the last column of zone k + 1)."""
    n, m, _ = B.shape
    w = 2 * m - 1
    N = n * m
    ab = np.zeros((2 * w + 1, N))
    for k in range(n):
        for blk, kc in ((A[k] if k > 0 else None, k - 1), (B[k], k), (C[k] if k + 1 < n else None, k + 1)):
            if blk is None:
                continue
            rows = k * m + np.arange(m)[:, None]
            cols = kc * m + np.arange(m)[None, :]
            ab[w + rows - cols, np.broadcast_to(cols, (m, m))] = blk
    return ab, w


def solve_ray(A, B, C, d) -> np.ndarray:
    """One ray by the banded LU of scipy (LAPACK gbsv)."""
    from scipy.linalg import solve_banded
    n, m, _ = B.shape
    if n == 0:
        return np.zeros((0, m))
    ab, w = band_storage(A, B, C)
    return solve_banded((w, w), ab, d.reshape(-1)).reshape(n, m)


def solve(A, B, C, d, offsets, rays=None) -> np.ndarray:
    """All rays (or the listed ones; other rows of the result stay NaN)."""
    Z, m = d.shape
    x = np.full((Z, m), np.nan)
    for r in (range(len(offsets) - 1) if rays is None else rays):
        a, b = int(offsets[r]), int(offsets[r + 1])
        x[a:b] = solve_ray(A[a:b], B[a:b], C[a:b], d[a:b])
    return x


def apply(A, B, C, x, offsets) -> np.ndarray:
    """The product M x ray by ray, from the blocks directly (A_k x_{k-1} + B_k x_k + C_k x_{k+1})."""
    y = np.einsum("zij,zj->zi", B, x)
    for r in range(len(offsets) - 1):
        a, b = int(offsets[r]), int(offsets[r + 1])
        if b - a > 1:
            y[a + 1:b] += np.einsum("zij,zj->zi", A[a + 1:b], x[a:b - 1])
            y[a:b - 1] += np.einsum("zij,zj->zi", C[a:b - 1], x[a + 1:b])
    return y
