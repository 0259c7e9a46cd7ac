"""FP64 reference transforms (test infrastructure only; see package docstring).

Layouts: sphere coefficients c[b, ig] (band-major, G order as given), cube
R[b, z, y, x] with x fastest (Sec. 2.1: n0 is the fastest dimension).
Grid extents n = (N0, N1, N2) for (x, y, z).

Conventions (Sec. 2.1 and 2.2):
  * G -> r uses e^{+j ...} and no scaling (psi(r) = sum_g c(g) e^{j g r});
  * r -> G uses omega_n = e^{-j 2 pi / n} and no scaling;
  * G sits at cube index (gx mod N0, gy mod N1, gz mod N2).
"""
from __future__ import annotations

import numpy as np


def _as_batch(c):
    c = np.asarray(c)
    return (c[None, :], True) if c.ndim == 1 else (c, False)


def _cube_index(gvec, n):
    g = np.asarray(gvec, dtype=np.int64)
    return (np.mod(g[:, 2], n[2]), np.mod(g[:, 1], n[1]), np.mod(g[:, 0], n[0]))


def g2r(gvec, c, n):
    """Zero-pad the sphere into the cube (Fig. 2), then the unnormalised
    inverse 3D DFT (Eq. 3dfft with the + sign of Sec. 2.2). numpy's pocketfft
    in double precision serves as the DFT step (norm="forward" leaves the
    inverse transform unscaled)."""
    c, squeeze = _as_batch(c)
    n0, n1, n2 = n
    cube = np.zeros((c.shape[0], n2, n1, n0), dtype=np.complex128)
    iz, iy, ix = _cube_index(gvec, n)
    cube[:, iz, iy, ix] = c
    out = np.fft.ifftn(cube, axes=(1, 2, 3), norm="forward")
    return out[0] if squeeze else out


def r2g(gvec, cube, n):
    """Unnormalised forward 3D DFT (omega_n = e^{-j 2 pi/n}, Sec. 2.1) of the
    cube, sampled at the sphere points."""
    cube = np.asarray(cube)
    squeeze = cube.ndim == 3
    if squeeze:
        cube = cube[None]
    spec = np.fft.fftn(cube.astype(np.complex128), axes=(1, 2, 3), norm="backward")
    iz, iy, ix = _cube_index(gvec, n)
    out = spec[:, iz, iy, ix]
    return out[0] if squeeze else out


def roundtrip(gvec, c, n):
    """G -> r -> G; equals N0 N1 N2 * c (no scaling in either direction)."""
    return r2g(gvec, g2r(gvec, c, n), n)


def apply_potential(gvec, c, v, n):
    """c' = P_sphere DFT_fwd(V * DFT_inv(pad(c))) (Sec. 2.3 fusion of pad,
    FFT and a pointwise product), unnormalised. v is real, shape (N2,N1,N0)."""
    v = np.asarray(v, dtype=np.float64)
    return r2g(gvec, g2r(gvec, c, n) * v, n)


def _phase(g, x, n):
    """exp(sign 2 pi j g x / n) argument with g*x reduced mod n first."""
    return 2.0 * np.pi * (np.mod(np.outer(g, x), n).astype(np.float64) / n)


def g2r_points(gvec, c, n, points):
    """Direct sum R[b, p] = sum_G c[b,G] exp(+2 pi j G.r_p / N) at chosen
    real-space points (P, 3) = (x, y, z). O(ngw) per point; this is the
    definition of Sec. 2.2 evaluated without any FFT."""
    c, squeeze = _as_batch(c)
    g = np.asarray(gvec, dtype=np.int64)
    p = np.asarray(points, dtype=np.int64)
    th = (_phase(g[:, 0], p[:, 0], n[0]) + _phase(g[:, 1], p[:, 1], n[1])
          + _phase(g[:, 2], p[:, 2], n[2]))            # (ngw, P)
    out = c.astype(np.complex128) @ np.exp(1j * th)
    return out[0] if squeeze else out


def r2g_points(gsel, cube, n):
    """Direct sum c[b, G] = sum_{x,y,z} R[b,z,y,x] exp(-2 pi j G.r / N) for
    selected G (P, 3). O(N0 N1 N2) per G; the definition of Sec. 2.1 / Eq.
    3dfft evaluated one output at a time."""
    cube = np.asarray(cube)
    squeeze = cube.ndim == 3
    if squeeze:
        cube = cube[None]
    n0, n1, n2 = n
    g = np.asarray(gsel, dtype=np.int64)
    ex = np.exp(-1j * _phase(g[:, 0], np.arange(n0), n0))   # (P, N0)
    ey = np.exp(-1j * _phase(g[:, 1], np.arange(n1), n1))   # (P, N1)
    ez = np.exp(-1j * _phase(g[:, 2], np.arange(n2), n2))   # (P, N2)
    out = np.empty((cube.shape[0], g.shape[0]), dtype=np.complex128)
    for i in range(g.shape[0]):
        t = cube.astype(np.complex128) @ ex[i]              # (B, N2, N1)
        t = t @ ey[i]                                       # (B, N2)
        out[:, i] = t @ ez[i]
    return out[0] if squeeze else out
