"""Sphere enumeration for the oracle (test infrastructure only).

Sec. 2.2: only plane waves with 1/2 |g|^2 <= E_cut are kept. Restated in grid
units with a k-shift: G integer, |G + k| <= r, inclusive. The squared distance
is evaluated left to right in IEEE double,
    d = ((gx+kx)*(gx+kx) + (gy+ky)*(gy+ky)) + (gz+kz)*(gz+kz),
without fused multiply-adds (numpy never fuses), and compared with r*r.

Canonical order (the CSR-over-xy offset array of Sec. 3.3 / Fig. 6, x fastest
as in Sec. 2.1): sorted by gy, then gx, then gz, each ascending over signed
values. A stick is one (gx, gy) column; its entries are contiguous.
"""
from __future__ import annotations

import numpy as np


def _axis_range(n: int) -> np.ndarray:
    """Signed frequencies of one axis: [-floor(n/2), n - floor(n/2))."""
    h = n // 2
    return np.arange(-h, n - h, dtype=np.int64)


def _in_ball(gx, gy, gz, k, radius):
    kx, ky, kz = (float(v) for v in k)
    ax = gx.astype(np.float64) + kx
    ay = gy.astype(np.float64) + ky
    az = gz.astype(np.float64) + kz
    d = ax * ax
    d = d + ay * ay
    d = d + az * az
    return d <= float(radius) * float(radius)


def sphere_fits(n, radius: float, k=(0.0, 0.0, 0.0)) -> bool:
    """True when every lattice point of the ball lies inside the grid range.

    The ball is enumerated over a box one cell wider than its extent on every
    side; a member outside [-N/2, N/2) on any axis would alias, so the plan
    is rejected.
    """
    r = float(radius)
    axes = []
    for d in range(3):
        kd = float(k[d])
        axes.append(np.arange(int(np.floor(-r - kd)) - 1,
                              int(np.ceil(r - kd)) + 2, dtype=np.int64))
    gx, gy, gz = np.meshgrid(*axes, indexing="ij")
    gx, gy, gz = gx.ravel(), gy.ravel(), gz.ravel()
    keep = _in_ball(gx, gy, gz, k, radius)
    for d, g in enumerate((gx[keep], gy[keep], gz[keep])):
        h = n[d] // 2
        if np.any(g < -h) or np.any(g >= n[d] - h):
            return False
    return True


def canonical_order(gvec: np.ndarray) -> np.ndarray:
    """Permutation that sorts (ngw, 3) rows by (gy, gx, gz)."""
    g = np.asarray(gvec)
    return np.lexsort((g[:, 2], g[:, 0], g[:, 1]))


def sphere_gvectors(n, radius: float, k=(0.0, 0.0, 0.0)) -> np.ndarray:
    """(ngw, 3) int32 array of (gx, gy, gz) in canonical order.

    Raises ValueError when the ball does not fit the grid (it would alias).
    """
    n = tuple(int(v) for v in n)
    if len(n) != 3 or min(n) < 1:
        raise ValueError("grid must have three positive extents")
    if not (radius >= 0.0):
        raise ValueError("radius must be non-negative")
    if not sphere_fits(n, radius, k):
        raise ValueError("sphere does not fit the grid")
    gx, gy, gz = np.meshgrid(_axis_range(n[0]), _axis_range(n[1]),
                             _axis_range(n[2]), indexing="ij")
    gx, gy, gz = gx.ravel(), gy.ravel(), gz.ravel()
    keep = _in_ball(gx, gy, gz, k, radius)
    g = np.stack([gx[keep], gy[keep], gz[keep]], axis=1)
    g = g[canonical_order(g)]
    return g.astype(np.int32)
