"""Error metric for comparing a GPU output with the oracle, row by row.

For every row (the last axis after moving `axis` there) with reference o, result g and magnitude
m (by default m = |o|; for a sum whose terms change sign, the same sum of absolute values, which
bounds its rounding):
  normwise     max|g - o| / max(m)
  elementwise  |g - o| / m on the entries with m >= 1e-3 max(m)
Rows whose magnitude lies entirely below the FP64 normal range are skipped (and counted).
"""
import numpy as np

TINY = 2.2250738585072014e-308


def row_errors(g, o, axis=-1, mag=None):
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, -1)
    o = np.moveaxis(np.asarray(o, dtype=np.float64), axis, -1)
    m = np.abs(o) if mag is None else np.moveaxis(np.asarray(mag, dtype=np.float64), axis, -1)
    n = o.shape[-1]
    g, o, m = g.reshape(-1, n), o.reshape(-1, n), m.reshape(-1, n)
    mx = np.max(m, axis=1)
    keep = mx >= TINY
    g, o, m, mx = g[keep], o[keep], m[keep], mx[keep]
    if len(mx) == 0:
        return 0.0, 0.0, int((~keep).sum())
    if not np.all(np.isfinite(g)):
        return np.inf, np.inf, int((~keep).sum())
    d = np.abs(g - o)
    nw = float(np.max(np.max(d, axis=1) / mx))
    big = m >= 1e-3 * mx[:, None]
    ew = float(np.max(np.where(big, d / np.where(big, m, 1.0), 0.0)))
    return nw, ew, int((~keep).sum())


def worst(g, o, axis=-1, mag=None):
    nw, ew, _ = row_errors(g, o, axis, mag)
    return max(nw, ew)


def magnitudes(ref):
    """Per-output magnitude arrays from an oracle result evaluated with mag=True."""
    out = {"j0": None, "chi0": None, "j1": ref.get("j1_abs"), "chi1": ref.get("chi1_abs")}
    if ref.get("phi_abs") is not None:
        out["phi"] = ref["phi_abs"]
    return out
