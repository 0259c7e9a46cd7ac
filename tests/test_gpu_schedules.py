"""Alternative radix schedules (64 = 16x4, 96 = 12x8, 128 = 8x16; the plane
stages of 160 = 40x4 with a composite 40-point DFT in registers and cube rows
fetched by bulk copies, its z lines 10x4x4; radix-10 and radix-12 codelets)
against the FP64 oracle, and the autotuner's choice among them."""
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


TUNE_FIELDS = ("chunk", "ctas0", "ctas1", "ctas2", "tiles", "level", "a_bufs", "sched_plane", "sched_stick", "pdl",
               "bg", "tc", "cl")


def tune_fields(line):
    """The fields of one tune-cache line (key, then the choice)."""
    assert len(line) == 1 + len(TUNE_FIELDS)
    return dict(zip(TUNE_FIELDS, (int(v) for v in line[1:])))


def relerr(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,r", [((64, 64, 64), 16.0), ((96, 96, 96), 24.0), ((128, 128, 128), 32.0),
                                 ((160, 160, 160), 40.0), ((64, 64, 96), 15.0)])
def test_alternative_schedules_roundtrip(F, n, r):
    import torch
    bands = 2
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    plan.set_radix_schedule(1, 1)
    assert plan.info["radix_schedule_plane"] == 7 and plan.info["radix_schedule_stick"] == 1
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 91).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    vol = n[0] * n[1] * n[2]
    c64 = c.astype(np.complex128)
    assert relerr(out.cpu().numpy(), vol * c64.reshape(-1)) <= 2e-6
    R = cube[:vol].view(n[2], n[1], n[0]).cpu().numpy().astype(np.complex128)
    assert relerr(R, oracle.g2r(g, c64[0], n)) <= 2e-6


def test_alternative_schedule_apply_and_r2g(F):
    import torch
    n, r = (96, 96, 96), 24.0
    g = oracle.sphere_gvectors(n, r)
    v = fi.gaussian_potential(n, 16, 4.0, seed=92).astype(np.float32)
    c = fi.complex_gaussian((3, len(g)), 93).astype(np.complex64)
    ap = F.Plan(n, "apply", "fp32", radius=r, bands=[3])
    ap.set_radix_schedule(1, 1)
    ap.set_potential(torch.from_numpy(v).cuda())
    out = torch.empty(c.size, dtype=torch.complex64, device="cuda")
    ap.execute(torch.from_numpy(c.reshape(-1)).cuda(), out)
    torch.cuda.synchronize()
    want = oracle.apply_potential(g, c.astype(np.complex128), v.astype(np.float64), n)
    assert relerr(out.cpu().numpy(), want) <= 2e-6
    R = fi.complex_gaussian((2, 96, 96, 96), 94).astype(np.complex64)
    p2 = F.Plan(n, "r2g", "fp32", radius=r, bands=[2])
    p2.set_radix_schedule(1, 1)
    o2 = torch.empty(p2.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    p2.execute(torch.from_numpy(R.reshape(-1)).cuda(), o2)
    torch.cuda.synchronize()
    assert relerr(o2.cpu().numpy(), oracle.r2g(g, R.astype(np.complex128), n).reshape(-1)) <= 2e-6


def test_schedule_errors_and_autotune(F, tmp_path, monkeypatch):
    import torch
    monkeypatch.setenv("FFTB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    p48 = F.Plan((48, 48, 48), "roundtrip", "fp32", radius=11.0, bands=[1])
    with pytest.raises(F.FFTBError) as ei:
        p48.set_radix_schedule(1, 0)
    assert ei.value.status == F.FFTB_ERR_UNSUPPORTED
    p64d = F.Plan((64, 64, 64), "roundtrip", "fp64", radius=16.0, bands=[1])
    with pytest.raises(F.FFTBError):
        p64d.set_radix_schedule(1, 0)
    with pytest.raises(F.FFTBError) as ei:
        p64d.set_radix_schedule(2, 0)
    assert ei.value.status == F.FFTB_ERR_INVALID_ARG
    # the autotuner may pick either schedule; the result stays correct and is cached
    n, r, bands = (128, 128, 128), 32.0, 6
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    plan.autotune(2)
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 95).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    assert relerr(out.cpu().numpy(), 128 ** 3 * c.reshape(-1).astype(np.complex128)) <= 2e-6
    line = (tmp_path / "tune.txt").read_text().strip().split()
    f = tune_fields(line)
    assert 0 <= f["sched_plane"] <= 3 and f["sched_stick"] in (0, 1) and f["pdl"] in (0, 1) and f["bg"] == 0
    assert f["tc"] == 0 and f["cl"] == 0  # an FP32 128-point plan has neither tensor-core nor cluster kernels
    assert f["sched_plane"] == plan.info["radix_schedule_plane"] and f["sched_stick"] == plan.info["radix_schedule_stick"]
    assert f["pdl"] == plan.info["dependent_launch"]


def test_160_two_pass_rows_by_bulk_copies(F):
    """The 160 = 40 x 4 plane schedule fetches each warp's next cube rows by
    bulk copies on a per-warp barrier: r -> G of random cubes against direct
    sums, from a 16-byte aligned cube (copies) and from a cube 8 bytes off
    (lane loads); then one copy withheld: the bounded wait runs out, the
    status is reported, and the next execute is correct."""
    import torch
    n, r, bands = (160, 160, 160), 40.0, 3
    vol = 160 ** 3
    plan = F.Plan(n, "r2g", "fp32", radius=r, bands=[bands])
    plan.set_radix_schedule(1, 0)
    g = plan.sphere(0)
    R = fi.complex_gaussian((bands, 160, 160, 160), 96).astype(np.complex64)
    sel = np.random.default_rng(97).choice(len(g), 5, replace=False)
    want = oracle.r2g_points(g[sel], R.astype(np.complex128), n)
    buf = torch.empty(bands * vol + 1, dtype=torch.complex64, device="cuda")
    out = torch.empty(plan.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    for off in (0, 1):  # 16-byte aligned, then 8 bytes off
        x = buf[off:off + bands * vol]
        x.copy_(torch.from_numpy(R.reshape(-1)))
        assert (x.data_ptr() % 16 == 0) == (off == 0)
        out.zero_()
        plan.execute(x, out)
        torch.cuda.synchronize()
        plan.check()
        got = out.cpu().numpy().reshape(bands, -1)[:, sel]
        assert relerr(got, want) <= 2e-6, off
        if off == 0:
            ref = out.clone()
    x = buf[:bands * vol]
    x.copy_(torch.from_numpy(R.reshape(-1)))
    plan.inject(F.FFTB_INJECT_SKIP_FIRST_PREFETCH)
    plan.execute(x, out)
    torch.cuda.synchronize()
    with pytest.raises(F.FFTBError) as ei:
        plan.check()
    assert ei.value.status == F.FFTB_ERR_DEVICE_TIMEOUT
    plan.inject(0)
    out.zero_()
    plan.execute(x, out)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(out, ref)


def test_160_two_pass_g2r_staged_sticks(F):
    """G -> r on the 160 = 40 x 4 plane schedule, whose y tasks take their
    sticks by bulk copies into the warps' exchange rows where each column's
    sticks are consecutive in gy: a canonical sphere with a k-point shift and
    a sphere with one whole stick taken out of a column (copies off for its
    planes), 2 + 3 bands in chunks of 2 that straddle the k-points, against
    the oracle; then one copy withheld: the bounded wait runs out, the status
    is reported, and the next execute is correct."""
    import torch
    n, r = (160, 160, 160), 40.0
    g0 = oracle.sphere_gvectors(n, r, (0.3, -0.2, 0.1))
    g1 = oracle.sphere_gvectors(n, r)
    g1 = g1[~((g1[:, 0] == 5) & (g1[:, 1] == 0))]  # a gap in the column x = 5
    plan = F.Plan(n, "g2r", "fp32", g_lists=[g0, g1], bands=[2, 3], max_chunk_bands=2)
    plan.set_radix_schedule(1, 0)
    assert plan.info["radix_schedule_plane"] & 1
    c = [fi.complex_gaussian((2, len(g0)), 98), fi.complex_gaussian((3, len(g1)), 99)]
    c = [a.astype(np.complex64) for a in c]
    x = torch.from_numpy(np.concatenate([a.reshape(-1) for a in c])).cuda()
    vol = 160 ** 3
    out = torch.empty(5 * vol, dtype=torch.complex64, device="cuda")
    plan.execute(x, out)
    torch.cuda.synchronize()
    plan.check()
    got = out.cpu().numpy().reshape(5, 160, 160, 160)
    want = [oracle.g2r(g0, c[0][b].astype(np.complex128), n) for b in range(2)]
    want += [oracle.g2r(g1, c[1][b].astype(np.complex128), n) for b in range(3)]
    for b in range(5):
        assert relerr(got[b], want[b]) <= 2e-6, b
    ref = out.clone()
    plan.inject(F.FFTB_INJECT_SKIP_FIRST_PREFETCH)
    plan.execute(x, out)
    torch.cuda.synchronize()
    with pytest.raises(F.FFTBError) as ei:
        plan.check()
    assert ei.value.status == F.FFTB_ERR_DEVICE_TIMEOUT
    plan.inject(0)
    out.zero_()
    plan.execute(x, out)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("r", [40.0, 41.0])
def test_160_two_pass_quarter_x_pruning(F, r):
    """The 160 = 40 x 4 plane kernels drop the middle half of each x line at
    compile time where every occupied x is within [-40, 40] (|G| <= 40), and
    run the whole line otherwise (|G| <= 41 reaches x = 41): round trip, the
    cube of a band and r -> G at sampled G against the oracle, and the fused
    apply against the oracle, in both cases."""
    import torch
    n, bands = (160, 160, 160), 2
    vol = 160 ** 3
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    plan.set_radix_schedule(1, 0)
    g = plan.sphere(0)
    assert (np.abs(g[:, 0]).max() <= 40) == (r == 40.0)
    assert plan.info["pruned_lines"] == (3 if r == 40.0 else 0)  # z stages, plane stages
    c = fi.complex_gaussian((bands, len(g)), 121).astype(np.complex64)
    c64 = c.astype(np.complex128)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()
    assert relerr(out.cpu().numpy(), vol * c64.reshape(-1)) <= 2e-6
    assert relerr(cube[vol:].view(160, 160, 160).cpu().numpy(), oracle.g2r(g, c64[1], n)) <= 2e-6
    del cube
    p2 = F.Plan(n, "r2g", "fp32", radius=r, bands=[1])
    p2.set_radix_schedule(1, 0)
    R = fi.complex_gaussian((160, 160, 160), 122).astype(np.complex64)
    o2 = torch.empty(p2.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    p2.execute(torch.from_numpy(R.reshape(-1)).cuda(), o2)
    torch.cuda.synchronize()
    p2.check()
    sel = np.random.default_rng(123).choice(len(g), 6, replace=False)
    sel[0] = int(np.argmax(np.abs(g[:, 0])))  # a G on the edge of the occupied x range
    assert relerr(o2.cpu().numpy()[sel], oracle.r2g_points(g[sel], R.astype(np.complex128), n)) <= 2e-6
    # a column with a gap: its sticks go through the scratch rows
    gg = g[~((g[:, 0] == -7) & (g[:, 1] == 3))]
    p3 = F.Plan(n, "r2g", "fp32", g_lists=[gg], bands=[1])
    p3.set_radix_schedule(1, 0)
    o3 = torch.empty(p3.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    p3.execute(torch.from_numpy(R.reshape(-1)).cuda(), o3)
    torch.cuda.synchronize()
    p3.check()
    s3 = np.random.default_rng(125).choice(len(gg), 6, replace=False)
    assert relerr(o3.cpu().numpy()[s3], oracle.r2g_points(gg[s3], R.astype(np.complex128), n)) <= 2e-6
    pa = F.Plan(n, "apply", "fp32", radius=r, bands=[1])
    pa.set_radix_schedule(1, 0)
    v = fi.gaussian_potential(n, 16, 5.0, seed=124).astype(np.float32)
    pa.set_potential(torch.from_numpy(v).cuda())
    oa = torch.empty(pa.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    pa.execute(torch.from_numpy(c[0].copy()).cuda(), oa)
    torch.cuda.synchronize()
    pa.check()
    assert relerr(oa.cpu().numpy(), oracle.apply_potential(g, c64[:1], v.astype(np.float64), n)) <= 2e-6


def test_160_two_pass_g2r_paired_store_paths(F):
    """The G -> r x lines of the 160 = 40 x 4 schedule own adjacent output
    pairs and store them as 16-byte pairs where the cube starts on a 16-byte
    boundary: a cube 8 bytes off that boundary takes the 8-byte stores (same
    values, bit for bit), and the batch-fastest cube (points B_k apart) is
    stored point by point; both against the oracle."""
    import torch
    n, r, bands = (160, 160, 160), 40.0, 2
    vol = 160 ** 3
    plan = F.Plan(n, "g2r", "fp32", radius=r, bands=[bands])
    plan.set_radix_schedule(1, 0)
    assert plan.info["radix_schedule_plane"] & 1
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 131).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty(bands * vol, dtype=torch.complex64, device="cuda")
    plan.execute(x, out)
    buf = torch.zeros(bands * vol + 1, dtype=torch.complex64, device="cuda")
    off = buf[1:]  # 8 bytes past a 16-byte boundary
    assert off.data_ptr() % 16 == 8
    plan.execute(x, off)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(off, out)
    assert buf[0].item() == 0
    got = out.view(bands, 160, 160, 160)[1].cpu().numpy()
    assert relerr(got, oracle.g2r(g, c[1].astype(np.complex128), n)) <= 2e-6
    del out, buf, off
    pb = F.Plan(n, "g2r", "fp32", radius=r, bands=[3], layout=1)
    pb.set_radix_schedule(1, 0)
    cb = fi.complex_gaussian((3, len(g)), 132).astype(np.complex64)
    ob = torch.empty(pb.info["cube_elems"], dtype=torch.complex64, device="cuda")
    pb.execute(torch.from_numpy(np.ascontiguousarray(cb.T).reshape(-1)).cuda(), ob)
    torch.cuda.synchronize()
    pb.check()
    band2 = ob.view(160, 160, 160, 3)[..., 2].cpu().numpy()
    assert relerr(band2, oracle.g2r(g, cb[2].astype(np.complex128), n)) <= 2e-6
    torch.cuda.empty_cache()
