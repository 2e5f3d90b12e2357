"""Error metric for comparing a GPU output with the oracle, row by row.

For every row (the last axis after moving `axis` there): the normwise error
max|g - o| / max|o|, and the elementwise relative error on the entries with |o| >= 1e-3 max|o|.
Rows whose reference lies entirely below the FP64 normal range are skipped (and counted).
"""
import numpy as np

TINY = 2.2250738585072014e-308


def row_errors(g, o, axis=-1):
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, -1)
    o = np.moveaxis(np.asarray(o, dtype=np.float64), axis, -1)
    n = o.shape[-1]
    g = g.reshape(-1, n)
    o = o.reshape(-1, n)
    m = np.max(np.abs(o), axis=1)
    keep = m >= TINY
    g, o, m = g[keep], o[keep], m[keep]
    if len(m) == 0:
        return 0.0, 0.0, int((~keep).sum())
    if not np.all(np.isfinite(g)):
        return np.inf, np.inf, int((~keep).sum())
    d = np.abs(g - o)
    nw = float(np.max(np.max(d, axis=1) / m))
    big = np.abs(o) >= 1e-3 * m[:, None]
    ew = float(np.max(np.where(big, d / np.where(big, np.abs(o), 1.0), 0.0)))
    return nw, ew, int((~keep).sum())


def worst(g, o, axis=-1):
    nw, ew, _ = row_errors(g, o, axis)
    return max(nw, ew)
