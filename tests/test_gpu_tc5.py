"""MIXED_TC plane stages on the 5th-generation tensor cores (tcgen05).

Grids 16, 32, 48 and 64 with N0 == N1 run their y- and x-DFTs as dense
split-FP16 products with FP32 accumulation in tensor memory; the rest of the
path is FP32. Every result is compared with the FP64 oracle at the
split-precision bound (relative L2 <= 1e-5).
"""
import numpy as np
import pytest

import fftb_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_2406_05577_gb300 import build
    build.build()
    from paper_2406_05577_gb300 import fftb
    assert torch.cuda.is_available()
    return fftb


def relerr(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).cuda()


CASES = [
    # grid, radius, k-shifts, bands per k-point
    ((16, 16, 16), 4.0, None, [3]),
    ((32, 32, 32), 8.0, None, [4]),
    ((48, 48, 48), 11.5, [(0.3, -0.2, 0.1), (-0.45, 0.4, -0.3)], [2, 5]),
    ((64, 64, 64), 16.0, None, [9]),
    ((64, 64, 32), 15.0, [(0.25, 0.25, -0.5)], [3]),
]


@pytest.mark.parametrize("n,r,ks,bands", CASES)
def test_tc5_roundtrip_vs_oracle(F, n, r, ks, bands):
    import torch
    kw = dict(radius=r, bands=bands)
    if ks is not None:
        kw["kshift"] = np.array(ks)
    plan = F.Plan(n, "roundtrip", "mixed", **kw)
    assert plan.info["tensor_core_planes"] == 3
    gs = [plan.sphere(k) for k in range(len(bands))]
    parts = [fi.complex_gaussian((b, len(g)), 500 + k).astype(np.complex64) for k, (g, b) in enumerate(zip(gs, bands))]
    x = dev(np.concatenate([p.reshape(-1) for p in parts]))
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()
    vol = n[0] * n[1] * n[2]
    assert relerr(out.cpu().numpy(), vol * x.cpu().numpy().astype(np.complex128)) <= TOL
    R = cube.cpu().numpy().astype(np.complex128)
    b0 = 0
    for k, (g, b) in enumerate(zip(gs, bands)):
        want = oracle.g2r(g, parts[k].astype(np.complex128), n)
        assert relerr(R[b0 * vol:(b0 + b) * vol].reshape(b, n[2], n[1], n[0]), want) <= TOL
        b0 += b


@pytest.mark.parametrize("n,r", [((32, 32, 32), 8.0), ((64, 64, 64), 16.0)])
def test_tc5_r2g_of_a_full_cube(F, n, r):
    """r -> G of a cube that is not band-limited: every x and y contributes."""
    import torch
    bands = 3
    plan = F.Plan(n, "r2g", "mixed", radius=r, bands=[bands])
    assert plan.info["tensor_core_planes"] == 3
    g = plan.sphere(0)
    R = fi.complex_gaussian((bands, n[2], n[1], n[0]), 61).astype(np.complex64)
    out = torch.empty(plan.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(dev(R), out)
    torch.cuda.synchronize()
    assert relerr(out.cpu().numpy(), oracle.r2g(g, R.astype(np.complex128), n).reshape(-1)) <= TOL


def test_tc5_g2r_wide_dynamic_range(F):
    """Bands whose sizes differ by 2^40 and planes of mixed magnitude: the
    per-plane power-of-two scaling keeps every band at the split-precision
    bound on its own."""
    import torch
    n, r, bands = (64, 64, 64), 16.0, 4
    plan = F.Plan(n, "g2r", "mixed", radius=r, bands=[bands])
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 62)
    c *= np.array([1e-12, 1.0, 1e6, 3e-3])[:, None]
    c = c.astype(np.complex64)
    out = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(dev(c), out)
    torch.cuda.synchronize()
    R = out.cpu().numpy().reshape(bands, 64, 64, 64).astype(np.complex128)
    want = oracle.g2r(g, c.astype(np.complex128), n)
    for b in range(bands):
        assert relerr(R[b], want[b]) <= TOL, b


def test_tc5_zero_band_and_unaligned_cube(F):
    """An all-zero band stays exactly zero; a cube 8 bytes off the 16-byte grid
    takes the non-bulk r -> G kernel and agrees with the oracle too."""
    import torch
    n, r, bands = (32, 32, 32), 8.0, 2
    plan = F.Plan(n, "roundtrip", "mixed", radius=r, bands=[bands])
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 63).astype(np.complex64)
    c[1] = 0
    x = dev(c)
    out = torch.empty_like(x)
    buf = torch.empty(plan.info["cube_elems"] + 1, dtype=torch.complex64, device="cuda")
    cube = buf[1:]
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(bands, -1)
    assert not np.any(o[1])
    assert relerr(o[0], 32 ** 3 * c[0].astype(np.complex128)) <= TOL


def test_tc5_bounded_wait_runs_out_and_is_reported(F):
    import torch
    n, r, bands = (32, 32, 32), 8.0, 3
    plan = F.Plan(n, "roundtrip", "mixed", radius=r, bands=[bands])
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 64).astype(np.complex64)
    x = dev(c)
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.inject(F.FFTB_INJECT_SKIP_FIRST_PREFETCH)
    plan.execute(x, out, cube)
    with pytest.raises(F.FFTBError) as ei:
        plan.check()
    assert ei.value.status == F.FFTB_ERR_DEVICE_TIMEOUT
    plan.inject(0)
    plan.execute(x, out, cube)
    plan.check()
    assert relerr(out.cpu().numpy(), 32 ** 3 * c.reshape(-1).astype(np.complex128)) <= TOL
