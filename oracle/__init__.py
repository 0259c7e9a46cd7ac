"""FP64 CPU oracle for the plane-wave sphere <-> cube 3D FFT.

TEST INFRASTRUCTURE ONLY. Nothing in the product library imports, links or
runs this package; only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may call it. It shares no code with the CUDA path.

What it computes (the plain definition, written out):

* sphere (Sec. 2.2, cutoff rule 1/2 |g|^2 <= E_cut): the integer G with
  |G + k| <= r, restated in grid units, components in [-N/2, N/2);
* G -> r (Sec. 2.2, psi(r) = sum_g c(g) e^{+j g r}):
  R[x,y,z] = sum_G c(G) exp(+2 pi j (gx x/N0 + gy y/N1 + gz z/N2)),
  i.e. the unnormalised inverse 3D DFT of the sphere zero-padded into the
  full cube (Fig. 2 full padding, which the staged padding of Fig. 3 equals);
* r -> G (Sec. 2.1, omega_n = e^{-j 2 pi / n}): the unnormalised forward 3D
  DFT (Eq. 3dfft) sampled at the sphere points;
* apply (Sec. 2.3, pad / FFT / pointwise product fused):
  c' = P_sphere DFT_fwd(V * DFT_inv(pad(c))).

Every function is pinned by ``tests/test_oracle_pins.py`` against brute-force
triple sums, closed forms (plane wave, delta), Parseval, the round trip
N0 N1 N2 * identity and published lattice-point counts.
"""
from .sphere import sphere_gvectors, sphere_fits, canonical_order
from .transform import (g2r, r2g, apply_potential, g2r_points, r2g_points,
                        roundtrip)

__all__ = [
    "sphere_gvectors", "sphere_fits", "canonical_order", "g2r", "r2g",
    "apply_potential", "g2r_points", "r2g_points", "roundtrip",
]
