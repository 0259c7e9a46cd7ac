"""Plans from the paper's other input descriptions: the whole frequency box
(the unpruned full-cube transform, Sec. 2.3 / Fig. 5) and an offset array
over a bounding domain (Sec. 3.3, Figs. 6-7), the latter also with the batch
dimension fastest as in Fig. 7. The box results are checked against numpy's
FFT of the zero-padded cube and the oracle, the rest against the oracle."""
import numpy as np
import pytest

import fftb_inputs as fi
import oracle

pytestmark = pytest.mark.gpu


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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dense(g, c, n):
    """coefficients c (bands, ngw) at G -> cube [bands][N2][N1][N0] (FFT wrap)"""
    cube = np.zeros((c.shape[0], n[2], n[1], n[0]), np.complex128)
    cube[:, g[:, 2] % n[2], g[:, 1] % n[1], g[:, 0] % n[0]] = c
    return cube


@pytest.mark.parametrize("n,prec", [((24, 24, 24), "fp64"), ((32, 32, 32), "fp32"), ((32, 32, 48), "fp32"),
                                    ((128, 128, 128), "fp32")])
def test_full_box_g2r_is_the_full_3d_fft(F, n, prec):
    import torch
    g = F.fftb_box_enumerate(n)
    bands = 1 if n[0] >= 128 else 2
    plan = F.Plan(n, "g2r", prec, g_lists=[g], bands=[bands])
    assert plan.info["max_sticks"] == n[0] * n[1] and plan.info["max_slabs"] == n[0]
    cd = np.complex128 if prec == "fp64" else np.complex64
    c = fi.complex_gaussian((bands, len(g)), 401).astype(cd)
    out = torch.empty(plan.info["cube_elems"], dtype=torch.complex128 if prec == "fp64" else torch.complex64,
                      device="cuda")
    plan.execute(torch.from_numpy(c.reshape(-1)).cuda(), out)
    torch.cuda.synchronize()
    vol = n[0] * n[1] * n[2]
    want = np.fft.ifftn(dense(g, c.astype(np.complex128), n), axes=(1, 2, 3)) * vol
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert relerr(out.cpu().numpy(), want) <= tol
    if n[0] <= 32:
        assert relerr(out.cpu().numpy(), oracle.g2r(g, c.astype(np.complex128), n)) <= tol


def test_full_box_256_all_slabs_occupied(F):
    """The whole 256^3 box (65 536 sticks, every one of the 256 x values an
    occupied slab, slab planes in device memory): G -> r of one band against
    the oracle, and the round trip of the box equals N0 N1 N2 times its
    input."""
    import torch
    n = (256, 256, 256)
    g = F.fftb_box_enumerate(n)
    plan = F.Plan(n, "roundtrip", "fp32", g_lists=[g], bands=[1])
    assert plan.info["max_sticks"] == 65536 and plan.info["max_slabs"] == 256
    c = fi.complex_gaussian((1, len(g)), 403).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()
    assert relerr(cube.cpu().numpy(), oracle.g2r(g, c[0].astype(np.complex128), n)) <= 2e-6
    vol = 256 ** 3
    assert relerr(out.cpu().numpy(), vol * c.reshape(-1).astype(np.complex128)) <= 2e-6


def test_full_box_r2g_and_roundtrip(F):
    import torch
    n = (64, 64, 64)
    g = F.fftb_box_enumerate(n)
    bands = 2
    R = fi.complex_gaussian((bands, n[2], n[1], n[0]), 402).astype(np.complex64)
    p = F.Plan(n, "r2g", "fp32", g_lists=[g], bands=[bands])
    out = torch.empty(bands * len(g), dtype=torch.complex64, device="cuda")
    p.execute(torch.from_numpy(R.reshape(-1)).cuda(), out)
    torch.cuda.synchronize()
    full = np.fft.fftn(R.astype(np.complex128), axes=(1, 2, 3))
    want = full[:, g[:, 2] % n[2], g[:, 1] % n[1], g[:, 0] % n[0]]
    assert relerr(out.cpu().numpy(), want) <= 2e-6
    rt = F.Plan(n, "roundtrip", "fp32", g_lists=[g], bands=[bands])
    c = fi.complex_gaussian((bands, len(g)), 403).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    o2 = torch.empty_like(x)
    cube = torch.empty(rt.info["cube_elems"], dtype=torch.complex64, device="cuda")
    rt.execute(x, o2, cube)
    torch.cuda.synchronize()
    assert relerr(o2.cpu().numpy(), 64 ** 3 * c.reshape(-1).astype(np.complex128)) <= 2e-6


@pytest.mark.parametrize("lo,hi,layout", [((0, 0, 0), (63, 63, 63), 1), ((-16, -16, -16), (16, 16, 16), 0),
                                          ((0, 0, 0), (63, 63, 63), 0)])
def test_offset_array_over_a_domain(F, lo, hi, layout):
    """Fig. 7's description: a 64^3 grid, the sphere of radius 16 given by the
    offset array over the domain, bands declared first (fastest) or last."""
    import torch
    n = (64, 64, 64)
    gs = oracle.sphere_gvectors(n, 16.0).astype(np.int64)
    lo_a, hi_a = np.asarray(lo), np.asarray(hi)
    v = lo_a + np.mod(gs - lo_a, 64)
    nx = hi_a[0] - lo_a[0] + 1
    col = (v[:, 1] - lo_a[1]) * nx + (v[:, 0] - lo_a[0])
    order = np.lexsort((v[:, 2], col))
    offsets = np.zeros(nx * (hi_a[1] - lo_a[1] + 1) + 1, np.int64)
    np.add.at(offsets, col + 1, 1)
    offsets = np.cumsum(offsets)
    g = F.fftb_glist_from_offsets(n, lo, hi, offsets, v[order, 2])
    assert np.array_equal(g, gs[order])
    bands = 4
    c = fi.complex_gaussian((bands, len(g)), 404).astype(np.complex64)
    x = c.T.reshape(-1) if layout == 1 else c.reshape(-1)
    plan = F.Plan(n, "g2r", "fp32", g_lists=[g], bands=[bands], layout=layout)
    out = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(torch.from_numpy(np.ascontiguousarray(x)).cuda(), out)
    torch.cuda.synchronize()
    R = out.cpu().numpy()
    R = np.moveaxis(R.reshape(64, 64, 64, bands), -1, 0) if layout == 1 else R.reshape(bands, 64, 64, 64)
    assert relerr(R, oracle.g2r(g, c.astype(np.complex128), n)) <= 2e-6
