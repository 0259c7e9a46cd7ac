"""Pins for the FP64 oracle: values fixed by mathematics, not by the oracle.

Each test pins a different way the oracle could be wrong:
  * brute-force triple sums on tiny non-cubic grids (sign, axis order,
    index wrap, k-shift);
  * closed forms: one plane wave, the G = 0 constant, a real-space delta;
  * invariants: Parseval, round trip = N0 N1 N2 * identity, linearity,
    conjugate symmetry, separability in any axis order;
  * the cutoff rule against published lattice-point counts (OEIS A000605)
    and an independent column-sum count;
  * planted mistakes (wrong sign, swapped axes) are caught by the pins.
"""
import math
import os

import numpy as np
import pytest

import fftb_inputs as fi
from oracle import (apply_potential, g2r, g2r_points, r2g, r2g_points,
                    roundtrip, sphere_gvectors)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

TINY = [
    ((4, 6, 5), 1.5, (0.0, 0.0, 0.0)),
    ((8, 8, 8), 3.0, (0.0, 0.0, 0.0)),
    ((12, 10, 9), 3.0, (0.25, -0.4, 0.1)),
    ((6, 9, 10), 2.2, (-0.5, 0.3, 0.45)),
]


def relerr(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def brute_g2r(gvec, c, n):
    """Explicit sum over G of c_G exp(+2 pi j (gx x/N0 + gy y/N1 + gz z/N2))."""
    n0, n1, n2 = n
    z, y, x = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    out = np.zeros((n2, n1, n0), dtype=np.complex128)
    for (gx, gy, gz), cg in zip(gvec.tolist(), c.tolist()):
        out += cg * np.exp(2j * np.pi * (gx * x / n0 + gy * y / n1 + gz * z / n2))
    return out


def brute_r2g(gvec, cube, n):
    n0, n1, n2 = n
    z, y, x = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    out = []
    for gx, gy, gz in gvec.tolist():
        w = np.exp(-2j * np.pi * (gx * x / n0 + gy * y / n1 + gz * z / n2))
        out.append((cube * w).sum())
    return np.array(out)


# ---------------------------------------------------------------- sphere rule

def test_lattice_counts_match_published_sequence():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sphere_lattice_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for r, count in ((int(a), int(b)) for a, b in rows):
        n = 2 * r + 2
        assert len(sphere_gvectors((n, n, n), float(r))) == count, r


@pytest.mark.parametrize("r,n", [(16, 64), (24, 96), (32, 128), (40, 160)])
def test_lattice_counts_column_sum(r, n):
    # independent count: for each (x, y) in the disc, 2*isqrt(r^2-x^2-y^2)+1 points
    expect = 0
    for x in range(-r, r + 1):
        for y in range(-r, r + 1):
            t = r * r - x * x - y * y
            if t >= 0:
                expect += 2 * math.isqrt(t) + 1
    assert len(sphere_gvectors((n, n, n), float(r))) == expect


@pytest.mark.parametrize("n,r,k", TINY)
def test_sphere_membership_bruteforce(n, r, k):
    g = sphere_gvectors(n, r, k)
    members = set()
    for gx in range(-(n[0] // 2), n[0] - n[0] // 2):
        for gy in range(-(n[1] // 2), n[1] - n[1] // 2):
            for gz in range(-(n[2] // 2), n[2] - n[2] // 2):
                if math.dist((gx + k[0], gy + k[1], gz + k[2]), (0, 0, 0)) <= r + 1e-12:
                    members.add((gx, gy, gz))
    assert set(map(tuple, g.tolist())) == members
    # canonical order: (gy, gx, gz) ascending
    keys = [(b, a, c) for a, b, c in g.tolist()]
    assert keys == sorted(keys)


def test_sphere_symmetric_at_gamma():
    g = sphere_gvectors((24, 24, 24), 6.0)
    s = set(map(tuple, g.tolist()))
    assert {(-a, -b, -c) for a, b, c in s} == s
    assert {(b, a, c) for a, b, c in s} == s
    assert {(c, b, a) for a, b, c in s} == s


def test_sphere_rejects_alias():
    with pytest.raises(ValueError):
        sphere_gvectors((24, 24, 24), 12.0)
    with pytest.raises(ValueError):
        sphere_gvectors((24, 24, 16), 8.5)
    assert len(sphere_gvectors((25, 25, 25), 12.0)) > 0


# ------------------------------------------------------------- transforms

@pytest.mark.parametrize("n,r,k", TINY)
def test_g2r_matches_bruteforce(n, r, k):
    g = sphere_gvectors(n, r, k)
    c = fi.complex_gaussian(len(g), seed=11)
    assert relerr(g2r(g, c, n), brute_g2r(g, c, n)) < 1e-13


@pytest.mark.parametrize("n,r,k", TINY)
def test_r2g_matches_bruteforce(n, r, k):
    g = sphere_gvectors(n, r, k)
    cube = fi.complex_gaussian((n[2], n[1], n[0]), seed=12)
    assert relerr(r2g(g, cube, n), brute_r2g(g, cube, n)) < 1e-13


@pytest.mark.parametrize("n,r,k", TINY)
def test_point_sums_match_bruteforce(n, r, k):
    g = sphere_gvectors(n, r, k)
    c = fi.complex_gaussian((2, len(g)), seed=13)
    pts = np.array([[0, 0, 0], [1, 2, 3], [n[0] - 1, n[1] - 1, n[2] - 1], [2, 0, 1]])
    pts = pts % np.array(n)
    full = np.stack([brute_g2r(g, c[b], n) for b in range(2)])
    got = g2r_points(g, c, n, pts)
    want = full[:, pts[:, 2], pts[:, 1], pts[:, 0]]
    assert relerr(got, want) < 1e-13
    cube = fi.complex_gaussian((2, n[2], n[1], n[0]), seed=14)
    sel = g[::3]
    want = np.stack([brute_r2g(sel, cube[b], n) for b in range(2)])
    assert relerr(r2g_points(sel, cube, n), want) < 1e-13


def test_single_plane_wave():
    n = (12, 10, 9)
    g = sphere_gvectors(n, 3.0)
    i = int(np.nonzero((g == [2, -1, 2]).all(axis=1))[0][0])
    c = np.zeros(len(g), complex)
    c[i] = 1.0
    R = g2r(g, c, n)
    z, y, x = np.meshgrid(np.arange(9), np.arange(10), np.arange(12), indexing="ij")
    expect = np.exp(2j * np.pi * (2 * x / 12 - 1 * y / 10 + 2 * z / 9))
    assert np.abs(R - expect).max() < 1e-14
    assert np.allclose(np.abs(R), 1.0)


def test_gamma_coefficient_is_constant():
    n = (8, 8, 8)
    g = sphere_gvectors(n, 3.0)
    c = np.where((g == 0).all(axis=1), 1.0 + 0j, 0j)
    assert np.abs(g2r(g, c, n) - 1.0).max() < 1e-15


def test_real_space_delta():
    n = (12, 10, 9)
    g = sphere_gvectors(n, 3.0, (0.2, 0.1, -0.3))
    cube = np.zeros((9, 10, 12), complex)
    r0 = (5, 7, 2)  # (x, y, z)
    cube[r0[2], r0[1], r0[0]] = 1.0
    got = r2g(g, cube, n)
    expect = np.exp(-2j * np.pi * (g[:, 0] * r0[0] / 12 + g[:, 1] * r0[1] / 10
                                   + g[:, 2] * r0[2] / 9))
    assert np.abs(got - expect).max() < 1e-14


@pytest.mark.parametrize("n,r,k", TINY)
def test_parseval_roundtrip_linearity(n, r, k):
    g = sphere_gvectors(n, r, k)
    vol = n[0] * n[1] * n[2]
    c = fi.complex_gaussian((3, len(g)), seed=15)
    R = g2r(g, c, n)
    assert abs((np.abs(R) ** 2).sum() - vol * (np.abs(c) ** 2).sum()) < 1e-11 * vol * (np.abs(c) ** 2).sum()
    assert relerr(roundtrip(g, c, n), vol * c) < 1e-14
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    assert relerr(g2r(g, a * c[0] + b * c[1], n), a * R[0] + b * R[1]) < 1e-14


def test_conjugate_symmetric_sphere_gives_real_cube():
    n = (12, 10, 9)
    g = sphere_gvectors(n, 3.0)
    c = fi.complex_gaussian(len(g), seed=16)
    index = {tuple(v): i for i, v in enumerate(g.tolist())}
    mirror = np.array([index[(-a, -b, -cc)] for a, b, cc in g.tolist()])
    c = 0.5 * (c + np.conj(c[mirror]))
    R = g2r(g, c, n)
    assert np.abs(R.imag).max() < 1e-13 * np.abs(R.real).max()


def test_separable_any_axis_order():
    n = (12, 10, 9)
    g = sphere_gvectors(n, 3.0, (0.1, 0.2, 0.3))
    c = fi.complex_gaussian(len(g), seed=17)
    ref = g2r(g, c, n)
    pad = np.zeros((9, 10, 12), complex)
    pad[g[:, 2] % 9, g[:, 1] % 10, g[:, 0] % 12] = c
    for order in [(2, 1, 0), (0, 1, 2), (1, 2, 0)]:
        t = pad
        for ax in order:
            t = np.fft.ifft(t, axis=ax) * t.shape[ax]
        assert relerr(t, ref) < 1e-14


# ------------------------------------------------------------------ apply

def test_apply_constant_potential():
    n = (8, 8, 8)
    g = sphere_gvectors(n, 3.0)
    c = fi.complex_gaussian((2, len(g)), seed=18)
    v = np.full((8, 8, 8), 0.75)
    assert relerr(apply_potential(g, c, v, n), 0.75 * 512 * c) < 1e-14


def test_apply_cosine_potential_shifts_coefficients():
    # V = cos(2 pi q.r/N) => c'(G) = N^3/2 (c(G-q) + c(G+q)), c = 0 off-sphere
    n = (12, 10, 9)
    q = (1, 2, -1)
    g = sphere_gvectors(n, 3.0)
    c = fi.complex_gaussian(len(g), seed=19)
    z, y, x = np.meshgrid(np.arange(9), np.arange(10), np.arange(12), indexing="ij")
    v = np.cos(2 * np.pi * (q[0] * x / 12 + q[1] * y / 10 + q[2] * z / 9))
    index = {tuple(t): i for i, t in enumerate(g.tolist())}
    expect = np.zeros(len(g), complex)
    for i, (a, b, cc) in enumerate(g.tolist()):
        for s in (+1, -1):
            j = index.get((a - s * q[0], b - s * q[1], cc - s * q[2]))
            if j is not None:
                expect[i] += 0.5 * 1080 * c[j]
    assert relerr(apply_potential(g, c, v, n), expect) < 1e-13


# ------------------------------------------------------- planted mistakes

def test_pins_catch_wrong_sign():
    n = (12, 10, 9)
    g = sphere_gvectors(n, 3.0, (0.25, -0.4, 0.1))
    c = fi.complex_gaussian(len(g), seed=20)
    pad = np.zeros((9, 10, 12), complex)
    pad[g[:, 2] % 9, g[:, 1] % 10, g[:, 0] % 12] = c
    wrong = np.fft.fftn(pad)  # e^{-j}: the wrong sign for G -> r
    assert relerr(wrong, brute_g2r(g, c, n)) > 0.5


def test_pins_catch_swapped_axes():
    # x and y exchanged in the cube index on a cubic grid (shapes agree)
    n = (8, 8, 8)
    g = sphere_gvectors(n, 3.0, (0.25, -0.4, 0.1))
    c = fi.complex_gaussian(len(g), seed=21)
    pad = np.zeros((8, 8, 8), complex)
    pad[g[:, 2] % 8, g[:, 0] % 8, g[:, 1] % 8] = c
    wrong = np.fft.ifftn(pad, norm="forward")
    assert relerr(wrong, brute_g2r(g, c, n)) > 0.5
    assert relerr(g2r(g, c, n), brute_g2r(g, c, n)) < 1e-13


def test_g2r_r2g_match_bruteforce_on_random_shapes():
    """The brute-force pins on random small grids (odd and even extents),
    radii, k-shifts and coefficients (hypothesis, where installed)."""
    hyp = pytest.importorskip("hypothesis")
    from hypothesis import given, settings, strategies as st

    ext = st.integers(3, 9)

    @settings(max_examples=40, deadline=None)
    @given(n=st.tuples(ext, ext, ext), frac=st.floats(0.0, 1.0), k=st.tuples(*[st.floats(-0.5, 0.5)] * 3),
           seed=st.integers(0, 2 ** 31 - 1))
    def check(n, frac, k, seed):
        # the largest ball that cannot alias: |G + k| <= r needs r + |k_d| < N_d / 2 - ... per axis
        rmax = min(n[d] // 2 - abs(k[d]) - 0.01 for d in range(3))
        if rmax <= 0:
            return
        r = frac * rmax
        try:
            g = sphere_gvectors(n, r, np.array(k))
        except ValueError:
            return  # a ball that would alias is rejected, which is tested elsewhere
        if not len(g):
            return
        rng = np.random.default_rng(seed)
        c = rng.standard_normal(len(g)) + 1j * rng.standard_normal(len(g))
        assert relerr(g2r(g, c, n), brute_g2r(g, c, n)) < 1e-13
        R = rng.standard_normal((n[2], n[1], n[0])) + 1j * rng.standard_normal((n[2], n[1], n[0]))
        assert relerr(r2g(g, R, n), brute_r2g(g, R, n)) < 1e-13

    check()


# ------------------------------------------- pins at the workload lengths

def _direct_g2r_at(gvec, c, n, pts):
    """Direct sum at chosen points, written independently of the oracle: the
    phase of G.r is reduced to an integer numerator mod N per axis before the
    division, so large G x products keep full FP64 accuracy."""
    g = np.asarray(gvec, dtype=np.int64)
    out = np.empty(len(pts), dtype=np.complex128)
    for i, (x, y, z) in enumerate(np.asarray(pts).tolist()):
        th = ((g[:, 0] * x) % n[0]) / n[0] + ((g[:, 1] * y) % n[1]) / n[1] + ((g[:, 2] * z) % n[2]) / n[2]
        out[i] = np.sum(c * np.exp(2j * np.pi * th))
    return out


def _direct_r2g_at(gsel, cube, n):
    """c(G) = sum over the whole cube of R exp(-2 pi j G.r/N), one G at a
    time, with the same integer phase reduction."""
    n0, n1, n2 = n
    z, y, x = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    out = []
    for gx, gy, gz in np.asarray(gsel).tolist():
        th = ((gx * x) % n0) / n0 + ((gy * y) % n1) / n1 + ((gz * z) % n2) / n2
        out.append(np.sum(cube * np.exp(-2j * np.pi * th)))
    return np.array(out)


@pytest.mark.parametrize("n,r,k", [((24, 24, 24), 6.0, (0.0, 0.0, 0.0)),
                                   ((64, 64, 64), 16.0, (0.0, 0.0, 0.0)),
                                   ((96, 96, 96), 24.0, (0.31, -0.44, 0.12)),
                                   ((128, 128, 128), 32.0, (0.0, 0.0, 0.0)),
                                   ((160, 160, 160), 40.0, (0.0, 0.0, 0.0))])
def test_library_fft_at_workload_lengths(n, r, k):
    """The oracle's FFT step (pocketfft through numpy) at the lengths the GPU
    path is measured on, whose factors 3 and 5 the tiny-grid pins do not all
    reach: sampled outputs of g2r / r2g against direct sums, and the oracle's
    own point-sum functions against the same direct sums."""
    g = sphere_gvectors(n, r, k)
    rng = np.random.default_rng(int(n[0]))
    c = rng.standard_normal(len(g)) + 1j * rng.standard_normal(len(g))
    pts = np.stack([rng.integers(0, n[d], 6) for d in range(3)], axis=1)
    pts[0] = (0, 0, 0)
    pts[1] = (n[0] - 1, n[1] // 2, 1)
    want = _direct_g2r_at(g, c, n, pts)
    R = g2r(g, c, n)
    assert relerr(R[pts[:, 2], pts[:, 1], pts[:, 0]], want) < 1e-12
    assert relerr(g2r_points(g, c, n, pts), want) < 1e-12
    cube = rng.standard_normal((n[2], n[1], n[0])) + 1j * rng.standard_normal((n[2], n[1], n[0]))
    sel = np.concatenate([g[:1], g[-1:], g[rng.choice(len(g), 2, replace=False)]])
    want = _direct_r2g_at(sel, cube, n)
    full = r2g(g, cube, n)
    index = {tuple(v): i for i, v in enumerate(g.tolist())}
    assert relerr(full[[index[tuple(v)] for v in sel.tolist()]], want) < 1e-12
    assert relerr(r2g_points(sel, cube, n), want) < 1e-12
