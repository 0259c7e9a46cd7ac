"""fftb_g2r_noalloc: the G -> r entry point for callers that cannot allocate
device memory (real-time hosts, programs whose device memory belongs to their
own allocator, libraries that must not grow their caller's footprint). It
keeps its scratch in static device arrays instead of a plan.

Checked through the C ABI against the plan-based fftb_execute on the same
inputs, within the FP32 tolerance the other tests use, on two calls in a row
with different spheres (so stale contents of the shared arrays would show);
against the FP64 oracle directly on whole bands, including a small sphere
with an odd stick count right after a large one; and for its size-limit
errors. Collected last so that a failure here stops a -x run only after
every other test has run.
"""
import numpy as np
import pytest

import fftb_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_2406_05577_gb300 import build
    build.build()
    from paper_2406_05577_gb300 import fftb
    assert torch.cuda.is_available()
    return fftb


def relerr(a, b):
    a, b = np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def plan_result(F, n, r, k, bands, x):
    import torch
    plan = F.Plan(n, "g2r", "fp32", radius=r, kshift=None if k is None else [k], bands=[bands])
    out = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def noalloc_result(F, n, r, k, bands, x):
    import torch
    out = torch.empty(bands * n[0] * n[1] * n[2], dtype=torch.complex64, device="cuda")
    s = torch.cuda.current_stream()
    F.fftb_g2r_noalloc(n, r, k, bands, x.data_ptr(), out.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_plan_on_two_calls_in_a_row(F):
    import torch
    cases = [
        # 90 bands of 64^3 need several passes through the static scratch
        ((64, 64, 64), 16.0, None, 90, 101),
        ((24, 24, 24), 6.0, (0.25, -0.4, 0.1), 5, 102),
    ]
    for n, r, k, bands, seed in cases:
        g = F.fftb_sphere_enumerate(n, r, k)
        c = fi.complex_gaussian((bands, len(g)), seed).astype(np.complex64)
        x = torch.from_numpy(c.reshape(-1)).cuda()
        want = plan_result(F, n, r, k, bands, x)
        got = noalloc_result(F, n, r, k, bands, x)
        assert relerr(got, want) <= TOL, (n, relerr(got, want))


def test_noalloc_against_the_oracle_large_then_small_sphere(F):
    """Whole bands against the FP64 oracle: two bands of the 160^3, |G| <= 40
    workload shape, then at once a 32^3 sphere of radius 3.1 with a k-shift
    (29 sticks, an odd number, far fewer than the call before left in the
    shared arrays)."""
    import torch
    cases = [((160, 160, 160), 40.0, None, 2, 103), ((32, 32, 32), 3.1, (0.3, 0.1, -0.2), 3, 104)]
    for n, r, k, bands, seed in cases:
        g = oracle.sphere_gvectors(n, r, k if k else (0.0, 0.0, 0.0))
        assert np.array_equal(F.fftb_sphere_enumerate(n, r, k), g)
        nst, _ = F.fftb_sphere_sticks(n, g)
        if n[0] == 32:
            assert nst == 29
        c = fi.complex_gaussian((bands, len(g)), seed).astype(np.complex64)
        x = torch.from_numpy(c.reshape(-1)).cuda()
        got = noalloc_result(F, n, r, k, bands, x).reshape(bands, -1)
        c64 = c.astype(np.complex128)
        for b in range(bands):
            assert relerr(got[b], oracle.g2r(g, c64[b], n)) <= TOL, (n, b)


def test_noalloc_rejects_sizes_beyond_its_arrays(F):
    import torch
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    y = torch.zeros(8, dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FFTBError) as e:
        # |G| <= 70 on 160^3: one band's stick buffer alone is above the scratch size
        F.fftb_g2r_noalloc((160, 160, 160), 70.0, None, 1, x.data_ptr(), y.data_ptr(), None)
    assert e.value.status == F.FFTB_ERR_UNSUPPORTED
    assert "FFTB_NOALLOC" in str(e.value)
    with pytest.raises(F.FFTBError) as e:
        # the tables of 60 000 bands of the 160^3 sphere are above the table array
        F.fftb_g2r_noalloc((160, 160, 160), 40.0, None, 60000, x.data_ptr(), y.data_ptr(), None)
    assert e.value.status == F.FFTB_ERR_UNSUPPORTED
    assert "60000 bands" in str(e.value)
    with pytest.raises(F.FFTBError) as e:
        F.fftb_g2r_noalloc((24, 24, 24), 6.0, None, 70000, x.data_ptr(), y.data_ptr(), None)
    assert e.value.status == F.FFTB_ERR_UNSUPPORTED
    with pytest.raises(F.FFTBError) as e:
        # |G| <= 46 on 256^3 (93 occupied x values): within the scratch and
        # table sizes, but its 256 x 93 slab plane does not fit in shared memory
        F.fftb_g2r_noalloc((256, 256, 256), 46.0, None, 1, x.data_ptr(), y.data_ptr(), None)
    assert e.value.status == F.FFTB_ERR_UNSUPPORTED
    assert "shared memory" in str(e.value)
