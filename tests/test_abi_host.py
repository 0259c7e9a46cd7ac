"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/fftb.h declares, enumerates spheres bit-exactly like the
oracle's independent enumerator, and rejects bad plans with status codes."""
import os
import re

import numpy as np
import pytest

import fftb_inputs as fi
from oracle import sphere_gvectors

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fftb():
    from paper_2406_05577_gb300 import build
    build.build()
    from paper_2406_05577_gb300 import fftb as mod
    return mod


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fftb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fftb_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(fftb):
    names = declared_functions()
    assert "fftb_plan_create" in names and "fftb_execute" in names
    lib = fftb.lib()
    for name in names:
        assert hasattr(lib, name), name
    # and the binding covers them with the same names
    assert set(names) <= set(fftb.EXPORTS)


@pytest.mark.parametrize("n,r", [((24, 24, 24), 6.0), ((64, 64, 64), 16.0), ((32, 32, 48), 10.0),
                                 ((20, 20, 40), 6.5), ((12, 12, 16), 3.0), ((160, 160, 160), 40.0)])
def test_sphere_matches_oracle_bit_exact(fftb, n, r):
    got = fftb.fftb_sphere_enumerate(n, r)
    want = sphere_gvectors(n, r)
    assert got.dtype == np.int32 and np.array_equal(got, want)


def test_kshift_spheres_match_oracle(fftb):
    ks = fi.kshifts(8, seed=3)
    counts = []
    for k in ks:
        got = fftb.fftb_sphere_enumerate((96, 96, 96), 24.0, k)
        want = sphere_gvectors((96, 96, 96), 24.0, k)
        assert np.array_equal(got, want)
        counts.append(len(got))
    assert len(set(counts)) > 1  # uneven sphere sizes across k-points


@pytest.mark.parametrize("n,r,sticks,slabs", [((24, 24, 24), 6.0, 113, 13), ((64, 64, 64), 16.0, 797, 33),
                                              ((128, 128, 128), 32.0, 3209, 65),
                                              ((160, 160, 160), 40.0, 5025, 81),
                                              ((256, 256, 256), 64.0, 12853, 129)])
def test_stick_and_slab_counts(fftb, n, r, sticks, slabs):
    g = sphere_gvectors(n, r)
    # independent count from the oracle's list
    assert len({(a, b) for a, b, _ in g.tolist()}) == sticks
    assert len({a for a, _, _ in g.tolist()}) == slabs
    assert fftb.fftb_sphere_sticks(n, g) == (sticks, slabs)


def test_explicit_list_errors(fftb):
    g = sphere_gvectors((24, 24, 24), 6.0)
    dup = np.concatenate([g, g[:1]])
    with pytest.raises(fftb.FFTBError) as e:
        fftb.fftb_sphere_sticks((24, 24, 24), dup)
    assert e.value.status == fftb.FFTB_ERR_INVALID_ARG and "duplicate" in str(e.value)
    bad = g.copy()
    bad[0] = [12, 0, 0]  # outside [-12, 12)
    with pytest.raises(fftb.FFTBError):
        fftb.fftb_sphere_sticks((24, 24, 24), bad)
    assert fftb.fftb_sphere_sticks((24, 24, 24), np.zeros((0, 3), np.int32)) == (0, 0)


def test_plan_errors_before_device(fftb):
    E = fftb.FFTBError
    # extents outside the compiled list take the generic path when their prime
    # factors are 2, 3 and 5 (N0, N1 <= 512, N2 <= 256); others are refused
    for n in ((64, 64, 49), (64, 77, 64), (520, 64, 64), (64, 64, 270)):
        with pytest.raises(E) as e:
            fftb.fftb_plan_create(n, "roundtrip", "fp32", radius=16.0)
        assert e.value.status == fftb.FFTB_ERR_UNSUPPORTED, n
    with pytest.raises(E) as e:
        fftb.fftb_plan_create((24, 24, 24), "roundtrip", "fp32", radius=12.0)  # aliases
    assert e.value.status == fftb.FFTB_ERR_INVALID_ARG
    with pytest.raises(E) as e:
        fftb.fftb_plan_create((24, 24, 24), "roundtrip", "fp32", radius=6.0, bands=[-1])
    assert e.value.status == fftb.FFTB_ERR_INVALID_ARG
    with pytest.raises(E) as e:
        fftb.fftb_plan_create((24, 24, 24), "roundtrip", "fp32", radius=6.0, layout=2)
    assert e.value.status == fftb.FFTB_ERR_INVALID_ARG
    with pytest.raises(E) as e:
        fftb.fftb_plan_create((24, 24, 24), 7, "fp32", radius=6.0)
    assert e.value.status == fftb.FFTB_ERR_INVALID_ARG
    g = sphere_gvectors((24, 24, 24), 6.0)
    with pytest.raises(E) as e:
        fftb.fftb_plan_create((24, 24, 24), "g2r", "fp64", g_lists=[np.concatenate([g, g[:2]])])
    assert "duplicate" in str(e.value)


def test_sphere_enumerate_rejects_alias(fftb):
    with pytest.raises(fftb.FFTBError):
        fftb.fftb_sphere_enumerate((24, 24, 24), 12.0)
    with pytest.raises(fftb.FFTBError):
        fftb.fftb_sphere_enumerate((24, 24, 16), 8.5)
    assert len(fftb.fftb_sphere_enumerate((25, 25, 25), 12.0)) == len(sphere_gvectors((25, 25, 25), 12.0))


def test_box_enumerate(fftb):
    """The whole frequency box: every component in [-N/2, N/2), each G once,
    sorted by gy, then gx, then gz (signed)."""
    for n in [(4, 6, 5), (12, 12, 16), (32, 32, 32)]:
        g = fftb.fftb_box_enumerate(n)
        assert g.shape == (n[0] * n[1] * n[2], 3)
        for d in range(3):
            h = n[d] // 2
            assert g[:, d].min() == -h and g[:, d].max() == n[d] - h - 1
        assert len({tuple(v) for v in g}) == len(g)
        assert np.array_equal(np.lexsort((g[:, 2], g[:, 0], g[:, 1])), np.arange(len(g)))
    small = np.zeros((63, 3), np.int32)  # one triple short
    st = fftb.lib().fftb_box_enumerate((fftb.ctypes.c_int32 * 3)(4, 4, 4), small.ctypes.data, 63)
    assert st == fftb.FFTB_ERR_INVALID_ARG and not small.any()


def _csr_of(g, n, lo, hi):
    """an offset array over the domain [lo, hi] for the G list g: domain
    coordinates are the frequencies shifted into [lo, hi] by multiples of N"""
    g = np.asarray(g, np.int64)
    lo, hi = np.asarray(lo), np.asarray(hi)
    v = lo + np.mod(g - lo, np.asarray(n))
    assert np.all(v <= hi)
    nx, ny = hi[0] - lo[0] + 1, hi[1] - lo[1] + 1
    col = (v[:, 1] - lo[1]) * nx + (v[:, 0] - lo[0])
    order = np.lexsort((v[:, 2], col))
    offsets = np.zeros(nx * ny + 1, np.int64)
    np.add.at(offsets, col + 1, 1)
    return np.cumsum(offsets), v[order, 2].astype(np.int32), g[order]


@pytest.mark.parametrize("n,r,lo,hi", [((24, 24, 24), 6.0, (0, 0, 0), (23, 23, 23)),
                                       ((24, 24, 24), 6.0, (-6, -6, -6), (6, 6, 6)),
                                       ((32, 32, 48), 9.5, (-16, 0, -24), (15, 31, 23)),
                                       ((20, 20, 40), 6.5, (-7, -7, 0), (7, 7, 39))])
def test_glist_from_offsets(fftb, n, r, lo, hi):
    """The paper's offset array over a bounding domain (z compressed per xy
    column, any lower corner): the G list comes back in the data's order."""
    g = sphere_gvectors(n, r)
    offsets, zi, want = _csr_of(g, n, lo, hi)
    got = fftb.fftb_glist_from_offsets(n, lo, hi, offsets, zi)
    assert got.dtype == np.int32 and np.array_equal(got, want)
    # the list holds the sphere once: as many sticks as the offset array has runs
    assert fftb.fftb_sphere_sticks(n, got)[0] == int(np.count_nonzero(np.diff(offsets)))


def test_glist_from_offsets_errors(fftb):
    n = (8, 8, 8)
    E = fftb.FFTBError
    ok_off = np.zeros(8 * 8 + 1, np.int64)
    ok_off[1:] = 1
    zi = np.zeros(1, np.int32)
    assert np.array_equal(fftb.fftb_glist_from_offsets(n, (0, 0, 0), (7, 7, 7), ok_off, zi), [[0, 0, 0]])
    assert np.array_equal(fftb.fftb_glist_from_offsets(n, (4, 0, 0), (11, 7, 7), ok_off, zi), [[-4, 0, 0]])
    with pytest.raises(E) as e:  # nine x values on an 8-point grid alias
        fftb.fftb_glist_from_offsets(n, (0, 0, 0), (8, 7, 7), np.zeros(9 * 8 + 1, np.int64), zi[:0])
    assert e.value.status == fftb.FFTB_ERR_INVALID_ARG
    bad = ok_off.copy()
    bad[5] = 2  # not non-decreasing
    with pytest.raises(E):
        fftb.fftb_glist_from_offsets(n, (0, 0, 0), (7, 7, 7), bad, np.zeros(2, np.int32))
    with pytest.raises(E):  # last offset != nnz
        fftb.fftb_glist_from_offsets(n, (0, 0, 0), (7, 7, 7), ok_off, np.zeros(2, np.int32))
    with pytest.raises(E):  # z outside the domain
        fftb.fftb_glist_from_offsets(n, (0, 0, 0), (7, 7, 3), ok_off, np.array([5], np.int32))


def test_scale_needs_a_plan(fftb):
    assert fftb.lib().fftb_plan_set_scale(None, 1.0, 1.0) == fftb.FFTB_ERR_INVALID_ARG
