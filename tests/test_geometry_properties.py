"""Property tests of the host index work (bit-exact by definition): random
grids, radii and k-shifts; the library's sphere enumeration against the
oracle's, its stick/slab counts against a count of the oracle's list, and
offset arrays over random bounding domains back to the same list."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import sphere_gvectors  # noqa: E402

SIZES = [12, 16, 20, 24, 32, 40, 48, 64]


@pytest.fixture(scope="module")
def fftb():
    from paper_2406_05577_gb300 import build
    build.build()
    from paper_2406_05577_gb300 import fftb as mod
    return mod


grids = st.tuples(st.sampled_from(SIZES), st.sampled_from(SIZES), st.sampled_from(SIZES))
shifts = st.tuples(*[st.floats(-0.5, 0.5, allow_nan=False, allow_infinity=False)] * 3)


@settings(max_examples=60, deadline=None)
@given(n=grids, frac=st.floats(0.0, 0.45), k=shifts)
def test_sphere_and_counts_match_the_oracle(fftb, n, frac, k):
    r = frac * (min(n) // 2 - 1)
    want = sphere_gvectors(n, r, np.array(k))
    got = fftb.fftb_sphere_enumerate(n, r, np.array(k))
    assert np.array_equal(got, want)
    if len(want):
        sticks, slabs = fftb.fftb_sphere_sticks(n, want)
        assert sticks == len({(int(a), int(b)) for a, b, _ in want})
        assert slabs == len({int(a) for a, _, _ in want})


@settings(max_examples=40, deadline=None)
@given(n=grids, frac=st.floats(0.05, 0.45), lo_off=st.tuples(*[st.integers(-3, 3)] * 3), data=st.data())
def test_offset_arrays_over_random_domains(fftb, n, frac, lo_off, data):
    r = frac * (min(n) // 2 - 1)
    g = sphere_gvectors(n, r).astype(np.int64)
    if not len(g):
        return
    # a bounding domain of full width per axis with a random lower corner
    lo = np.array([-(n[d] // 2) + lo_off[d] for d in range(3)])
    hi = lo + np.array(n) - 1
    v = lo + np.mod(g - lo, np.array(n))
    nx = hi[0] - lo[0] + 1
    col = (v[:, 1] - lo[1]) * nx + (v[:, 0] - lo[0])
    order = np.lexsort((v[:, 2], col))
    offsets = np.zeros(nx * (hi[1] - lo[1] + 1) + 1, np.int64)
    np.add.at(offsets, col + 1, 1)
    got = fftb.fftb_glist_from_offsets(n, lo, hi, np.cumsum(offsets), v[order, 2].astype(np.int32))
    assert np.array_equal(got, g[order])
