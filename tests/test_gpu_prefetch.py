"""Plane kernels whose inputs arrive by bulk asynchronous copies (prefetch).

The prefetching kernels do the same arithmetic as the plain ones, so their
outputs must agree bit for bit; both are also checked against the FP64
oracle. The bounded waits are tested by withholding one copy on the host's
request: the wait runs out, the kernel leaves and the plan reports
FFTB_ERR_DEVICE_TIMEOUT, and the next execute is correct again.
"""
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


def run(plan, x, direction, cube_offset=0):
    import torch
    info = plan.info
    out_n = info["cube_elems"] if direction == "g2r" else info["sphere_elems"]
    out = torch.full((out_n,), float("nan"), dtype=x.dtype, device="cuda")
    cube = None
    if direction == "roundtrip":
        cube = torch.empty(info["cube_elems"], dtype=x.dtype, device="cuda")
    if cube_offset:
        # the same data one element (8 bytes) further on: rows off the 16-byte grid
        buf = torch.empty(x.numel() + cube_offset, dtype=x.dtype, device="cuda")
        buf[cube_offset:] = x
        x = buf[cube_offset:]
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    return out.cpu().numpy(), (cube.cpu().numpy() if cube is not None else None)


PREFETCH_CASES = [
    # grid, radius, k-shifts, bands per k
    ((64, 64, 64), 16.0, None, [8]),
    ((96, 96, 96), 24.0, [(0.1, -0.3, 0.2), (-0.45, 0.25, 0.0)], [3, 6]),
    ((128, 128, 128), 32.0, None, [2]),
    ((24, 24, 24), 6.0, None, [5]),
]


@pytest.mark.parametrize("n,r,ks,bands", PREFETCH_CASES)
def test_prefetch_roundtrip_matches_plain_and_oracle(F, n, r, ks, bands):
    import torch
    kw = dict(radius=r, bands=bands)
    if ks is not None:
        kw["kshift"] = np.array(ks)
    plan = F.Plan(n, "roundtrip", "fp32", **kw)
    # wherever the staging fits: G -> r at every size, r -> G where each warp
    # gets an x task per plane (grids of 64 and up)
    plan.set_prefetch(2)
    assert plan.info["prefetch"] & 1
    if n[0] >= 64:
        assert plan.info["prefetch"] & 2
    gs = [plan.sphere(k) for k in range(len(bands))]
    parts = [fi.complex_gaussian((b, len(g)), 40 + k).astype(np.complex64) for k, (g, b) in enumerate(zip(gs, bands))]
    x = torch.from_numpy(np.concatenate([p.reshape(-1) for p in parts])).cuda()
    out_pf, cube_pf = run(plan, x, "roundtrip")
    plan.set_prefetch(0)
    assert plan.info["prefetch"] == 0
    out_plain, cube_plain = run(plan, x, "roundtrip")
    assert np.array_equal(out_pf, out_plain)
    assert np.array_equal(cube_pf, cube_plain)
    vol = n[0] * n[1] * n[2]
    xs = x.cpu().numpy().astype(np.complex128)
    assert relerr(out_pf, vol * xs) <= 2e-6
    b0 = 0
    for k, (g, b) in enumerate(zip(gs, bands)):
        want = oracle.g2r(g, parts[k][0].astype(np.complex128), n)
        got = cube_pf[b0 * vol:(b0 + 1) * vol].reshape(n[2], n[1], n[0])
        assert relerr(got, want) <= 2e-6
        b0 += b


def test_prefetch_r2g_and_apply_vs_oracle(F):
    import torch
    n, r = (64, 64, 64), 16.0
    g = oracle.sphere_gvectors(n, r)
    R = fi.complex_gaussian((3, 64, 64, 64), 51).astype(np.complex64)
    plan = F.Plan(n, "r2g", "fp32", radius=r, bands=[3])
    assert plan.info["prefetch"] & 2
    xr = torch.from_numpy(R.reshape(-1)).cuda()
    got, _ = run(plan, xr, "r2g")
    want = np.concatenate([oracle.r2g(g, R[b].astype(np.complex128), n) for b in range(3)])
    assert relerr(got, want) <= 2e-6
    plan.set_prefetch(0)
    plain, _ = run(plan, xr, "r2g")
    assert np.array_equal(got, plain)

    v = fi.gaussian_potential(n, 16, 3.0, seed=52).astype(np.float32)
    c = fi.complex_gaussian((4, len(g)), 53).astype(np.complex64)
    ap = F.Plan(n, "apply", "fp32", radius=r, bands=[4])
    assert ap.info["prefetch"] & 4
    ap.set_potential(torch.from_numpy(v).cuda())
    xc = torch.from_numpy(c.reshape(-1)).cuda()
    got, _ = run(ap, xc, "apply")
    want = oracle.apply_potential(g, c.astype(np.complex128), v.astype(np.float64), n)
    assert relerr(got, want) <= 2e-6
    ap.set_prefetch(0)
    plain, _ = run(ap, xc, "apply")
    assert np.array_equal(got, plain)


def test_unaligned_cube_uses_plain_loads(F):
    """A cube that starts 8 bytes off a 16-byte boundary cannot be bulk-copied by
    rows: r -> G then runs the plain kernel, with the same result."""
    import torch
    n, r = (64, 64, 64), 16.0
    R = fi.complex_gaussian((2, 64, 64, 64), 61).astype(np.complex64)
    plan = F.Plan(n, "r2g", "fp32", radius=r, bands=[2])
    xr = torch.from_numpy(R.reshape(-1)).cuda()
    aligned, _ = run(plan, xr, "r2g")
    shifted, _ = run(plan, xr, "r2g", cube_offset=1)
    assert np.array_equal(aligned, shifted)


def test_no_prefetch_for_fp64_and_mixed(F):
    for prec in ("fp64", "mixed"):
        plan = F.Plan((64, 64, 64), "roundtrip", prec, radius=16.0, bands=[1])
        assert plan.info["prefetch"] == 0


def test_bounded_wait_runs_out_and_is_reported(F):
    """One copy withheld: the wait gives up after about a second, the status word
    is set, fftb_plan_check and fftb_execute_host report it, and the plan (and
    the CUDA context) work normally afterwards."""
    import torch
    n, r, bands = (64, 64, 64), 16.0, 4
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    assert plan.info["prefetch"] & 3
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 71).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    plan.check()  # nothing pending
    plan.inject(F.FFTB_INJECT_SKIP_FIRST_PREFETCH)
    run(plan, x, "roundtrip")
    with pytest.raises(F.FFTBError) as ei:
        plan.check()
    assert ei.value.status == F.FFTB_ERR_DEVICE_TIMEOUT
    plan.check()  # cleared by the previous check
    # the host-buffer entry point reports it from its own synchronisation
    host_in = c.reshape(-1).copy()
    host_out = np.empty_like(host_in)
    with pytest.raises(F.FFTBError) as ei:
        F.fftb_execute_host(plan.handle, host_in.ctypes.data, host_out.ctypes.data)
    assert ei.value.status == F.FFTB_ERR_DEVICE_TIMEOUT
    # injection off: correct again, nothing reported
    plan.inject(0)
    out, _ = run(plan, x, "roundtrip")
    plan.check()
    assert relerr(out, 64 ** 3 * c.reshape(-1).astype(np.complex128)) <= 2e-6
    F.fftb_execute_host(plan.handle, host_in.ctypes.data, host_out.ctypes.data)
    assert relerr(host_out, 64 ** 3 * c.reshape(-1).astype(np.complex128)) <= 2e-6
    with pytest.raises(F.FFTBError):
        plan.inject(8)
    with pytest.raises(F.FFTBError):
        plan.set_prefetch(3)


def test_slab_buffers_same_results(F):
    """One or two slab planes per CTA change only the schedule: bit-identical."""
    import torch
    n, r = (96, 96, 96), 24.0
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[5])
    plan.set_slab_buffers(2)
    assert plan.info["slab_buffers"] == 2
    g = plan.sphere(0)
    c = fi.complex_gaussian((5, len(g)), 81).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out2, cube2 = run(plan, x, "roundtrip")
    plan.set_slab_buffers(1)
    assert plan.info["slab_buffers"] == 1
    for level in (0, 2):
        plan.set_prefetch(level)
        out1, cube1 = run(plan, x, "roundtrip")
        assert np.array_equal(out1, out2) and np.array_equal(cube1, cube2)
    assert relerr(cube2[:96 ** 3].reshape(96, 96, 96), oracle.g2r(g, c[0].astype(np.complex128), n)) <= 2e-6
    with pytest.raises(F.FFTBError) as ei:
        plan.set_slab_buffers(3)
    assert ei.value.status == F.FFTB_ERR_INVALID_ARG
    big = F.Plan((160, 160, 160), "g2r", "fp32", radius=40.0, bands=[1])
    assert big.info["slab_buffers"] == 1  # two do not fit
    with pytest.raises(F.FFTBError) as ei:
        big.set_slab_buffers(2)
    assert ei.value.status == F.FFTB_ERR_UNSUPPORTED


def test_interleaved_plans_of_one_grid(F):
    """Plans of one grid with different spheres need different shared memory in
    the same kernels; creating the smaller one must not break the larger."""
    import torch
    n = (64, 64, 64)
    big = F.Plan(n, "g2r", "fp32", radius=16.0, bands=[2])
    small = F.Plan(n, "g2r", "fp32", radius=6.0, bands=[2])
    small.set_slab_buffers(1)
    for plan, seed in ((big, 91), (small, 92), (big, 93)):
        g = plan.sphere(0)
        c = fi.complex_gaussian((2, len(g)), seed).astype(np.complex64)
        out, _ = run(plan, torch.from_numpy(c.reshape(-1)).cuda(), "g2r")
        want = oracle.g2r(g, c.astype(np.complex128), n)
        assert relerr(out, want) <= 2e-6


@pytest.mark.parametrize("n,r,prec,sched", [((64, 64, 64), 16.0, "fp32", None), ((96, 96, 96), 24.0, "fp32", (1, 1)),
                                            ((32, 32, 32), 8.0, "fp64", None), ((64, 64, 64), 16.0, "mixed", None),
                                            ((128, 128, 128), 32.0, "fp32", None)])
def test_dependent_launch_same_results(F, n, r, prec, sched):
    """Programmatic dependent launch only lets each stage kernel start early and
    wait for its predecessor in the prologue: results are bit-identical to
    plainly ordered launches, across several executes of one graph."""
    import torch
    bands = 3
    plan = F.Plan(n, "roundtrip", prec, radius=r, bands=[bands])
    if sched is not None:
        plan.set_radix_schedule(*sched)
    g = plan.sphere(0)
    cd = np.complex128 if prec == "fp64" else np.complex64
    c = fi.complex_gaussian((bands, len(g)), 83).astype(cd)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    assert plan.info["dependent_launch"] == 1
    plan.set_pdl(False)
    assert plan.info["dependent_launch"] == 0
    out0, cube0 = run(plan, x, "roundtrip")
    plan.set_pdl(True)
    for _ in range(3):
        out1, cube1 = run(plan, x, "roundtrip")
        assert np.array_equal(out0, out1) and np.array_equal(cube0, cube1)
    plan.check()
    vol = n[0] * n[1] * n[2]
    tol = 1e-12 if prec == "fp64" else (1e-5 if prec == "mixed" else 2e-6)
    assert relerr(cube1[:vol].reshape(n[2], n[1], n[0]), oracle.g2r(g, c[0].astype(np.complex128), n)) <= tol


def test_prefetch_with_global_slab_planes(F):
    """256^3 keeps its slab planes in global memory; the prefetching plane
    kernels of that variant give the plain kernels' results bit for bit."""
    import torch
    n, r, bands = (256, 256, 256), 64.0, 2
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    assert plan.info["slab_planes_global"] == 1
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 85).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    plan.set_prefetch(2)
    assert plan.info["prefetch"] & 2  # r -> G at least (its staging is small)
    out_pf, cube_pf = run(plan, x, "roundtrip")
    plan.check()
    plan.set_prefetch(0)
    assert plan.info["prefetch"] == 0
    out0, cube0 = run(plan, x, "roundtrip")
    assert np.array_equal(out_pf, out0) and np.array_equal(cube_pf, cube0)
    assert relerr(out_pf, 256 ** 3 * c.reshape(-1).astype(np.complex128)) <= 2e-6


def test_global_slab_planes_one_or_two_buffers(F):
    """Plans whose slab planes live in global memory start with one buffer per
    CTA and may switch to two (the allocation holds both): same results."""
    import torch
    n, r, bands = (256, 256, 256), 64.0, 1
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    assert plan.info["slab_planes_global"] == 1 and plan.info["slab_buffers"] == 1
    g = plan.sphere(0)
    x = torch.from_numpy(fi.complex_gaussian((bands, len(g)), 86).astype(np.complex64).reshape(-1)).cuda()
    out1, cube1 = run(plan, x, "roundtrip")
    plan.set_slab_buffers(2)
    assert plan.info["slab_buffers"] == 2
    out2, cube2 = run(plan, x, "roundtrip")
    plan.check()
    assert np.array_equal(out1, out2) and np.array_equal(cube1, cube2)
