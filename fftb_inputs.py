"""Seeded synthetic inputs for the sphere <-> cube transform.

This module only draws random numbers and builds input arrays. It holds none
of the transform's arithmetic, so both the CUDA path and the CPU oracle can be
fed bit-identical inputs from it.

Recipes (plane-wave DFT workloads, Sec. 2.2 of the paper; no dataset exists):
  * coefficients c_b(G): i.i.d. complex Gaussian, real and imaginary parts each
    N(0, 1), from numpy's PCG64 ``default_rng(seed)`` (or one stream per band,
    ``default_rng([seed, band])``, for batches sharded across ranks);
  * optional envelope exp(-|G|^2 / (2 sigma^2)) (sigma = 8 grid units for the
    64^3 round-trip workload);
  * k-shifts uniform in [-0.5, 0.5)^3 grid units;
  * band counts per k-point uniform in an integer range;
  * local potential V(r): a sum of Gaussians with seeded centres in [0, N)^3,
    amplitudes in [-1, 1] and a periodic minimum-image distance.
"""
from __future__ import annotations

import numpy as np

# The five workloads: grid, cutoff radius, bands, precision, direction.
WORKLOADS = {
    "sphere24_fp64": dict(n=(24, 24, 24), radius=6.0, bands=4, seed=1,
                          precision="fp64", direction="both"),
    "sphere64_rt_fp32": dict(n=(64, 64, 64), radius=16.0, bands=64, seed=2,
                             precision="fp32", direction="roundtrip",
                             envelope_sigma=8.0),
    "sphere96_multik_fp32": dict(n=(96, 96, 96), radius=24.0, n_kpoints=8,
                                 bands_range=(16, 128), seed=3,
                                 precision="fp32", direction="roundtrip"),
    "sphere128_apply": dict(n=(128, 128, 128), radius=32.0, bands=256, seed=4,
                            precision="fp32", direction="apply",
                            n_gaussians=32, gaussian_width=4.0),
    "sphere160_large": dict(n=(160, 160, 160), radius=40.0, bands=512, seed=5,
                            precision="fp32", direction="both"),
}


def complex_gaussian(shape, seed: int) -> np.ndarray:
    """complex128 array whose real and imaginary parts are i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def complex_gaussian_bands(first: int, count: int, ngw: int, seed: int) -> np.ndarray:
    """Bands first .. first + count - 1 of a batch of sphere coefficients,
    (count, ngw) complex128, where band i is drawn from its own stream
    default_rng([seed, i]) (ngw real parts, then ngw imaginary parts, each
    N(0, 1)): a contiguous slice of the batch is the same whichever process
    draws it, so ranks that each draw their shard hold one global batch."""
    out = np.empty((count, ngw), dtype=np.complex128)
    for j in range(count):
        rng = np.random.default_rng([seed, first + j])
        out[j].real = rng.standard_normal(ngw)
        out[j].imag = rng.standard_normal(ngw)
    return out


def gaussian_envelope(gvec: np.ndarray, sigma: float) -> np.ndarray:
    """exp(-|G|^2 / (2 sigma^2)) for each row of an (ngw, 3) integer array."""
    g = np.asarray(gvec, dtype=np.float64)
    g2 = (g * g).sum(axis=1)
    return np.exp(-g2 / (2.0 * sigma * sigma))


def kshifts(n_kpoints: int, seed: int) -> np.ndarray:
    """(n_kpoints, 3) float64 shifts, uniform in [-0.5, 0.5)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.5, 0.5, size=(n_kpoints, 3))


def band_counts(n_kpoints: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """(n_kpoints,) int32 band counts, uniform in [lo, hi] inclusive."""
    rng = np.random.default_rng(seed + 1000)
    return rng.integers(lo, hi + 1, size=n_kpoints).astype(np.int32)


def gaussian_potential(n, n_gaussians: int, width: float, seed: int) -> np.ndarray:
    """Real potential V on the grid, shape (N2, N1, N0), x fastest.

    V(r) = sum_i a_i exp(-d_i(r)^2 / (2 width^2)), centres u_i uniform in
    [0, N)^3, amplitudes a_i uniform in [-1, 1], d_i the periodic
    minimum-image distance. Built in float64.
    """
    n0, n1, n2 = n
    rng = np.random.default_rng(seed + 2000)
    centres = rng.uniform(0.0, 1.0, size=(n_gaussians, 3)) * np.array([n0, n1, n2])
    amps = rng.uniform(-1.0, 1.0, size=n_gaussians)
    x = np.arange(n0, dtype=np.float64)
    y = np.arange(n1, dtype=np.float64)
    z = np.arange(n2, dtype=np.float64)
    v = np.zeros((n2, n1, n0), dtype=np.float64)

    def mi(d, L):
        d = np.abs(d)
        return np.minimum(d, L - d)

    for (ux, uy, uz), a in zip(centres, amps):
        dx = mi(x - ux, n0)
        dy = mi(y - uy, n1)
        dz = mi(z - uz, n2)
        d2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        v += a * np.exp(-d2 / (2.0 * width * width))
    return v
