"""Full-size workloads on the GPU, in the launch configuration the benchmark
times: checked on sampled outputs the oracle computes one by one (direct
sums), and on properties that hold at any size (round trip = N0 N1 N2 * c,
Parseval). A few whole bands are also compared with the full oracle."""
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def sample_points(n, count, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, n[0], count), rng.integers(0, n[1], count),
                     rng.integers(0, n[2], count)], axis=1)


def test_roundtrip_64_full_batch_fp32(F):
    """64^3, |G| <= 16, 64 bands, FP32, envelope exp(-|G|^2/(2*64)): the bench workload."""
    import torch
    n, r, bands = (64, 64, 64), 16.0, 64
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    g = plan.sphere(0)
    assert len(g) == 17077
    c = fi.complex_gaussian((bands, len(g)), 2) * fi.gaussian_envelope(g, 8.0)[None, :]
    c = c.astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    c64 = c.astype(np.complex128)
    back = out.cpu().numpy().astype(np.complex128).reshape(bands, -1)
    assert relerr(back, 64 ** 3 * c64) <= 2e-6
    R = cube.view(bands, 64, 64, 64).cpu().numpy().astype(np.complex128)
    # whole bands against the full oracle
    for b in (0, 37, 63):
        assert relerr(R[b], oracle.g2r(g, c64[b], n)) <= 2e-6
    # sampled points of every band against direct sums
    pts = sample_points(n, 24, 3)
    want = oracle.g2r_points(g, c64, n, pts)
    got = R[:, pts[:, 2], pts[:, 1], pts[:, 0]]
    assert relerr(got, want) <= 2e-6
    # Parseval per band
    e_r = (np.abs(R) ** 2).sum(axis=(1, 2, 3))
    e_g = 64 ** 3 * (np.abs(c64) ** 2).sum(axis=1)
    assert np.max(np.abs(e_r / e_g - 1)) < 1e-5


def test_apply_128_fp32_and_fp64(F):
    """128^3, |G| <= 32, V = 32 Gaussians of width 4: 8 bands against the full oracle."""
    import torch
    n, r, bands = (128, 128, 128), 32.0, 8
    v = fi.gaussian_potential(n, 32, 4.0, seed=4)
    g = oracle.sphere_gvectors(n, r)
    c = fi.complex_gaussian((bands, len(g)), 4)
    for prec, tol in (("fp32", 2e-6), ("fp64", 1e-12)):
        plan = F.Plan(n, "apply", prec, radius=r, bands=[bands])
        vr = v.astype(np.float32 if prec == "fp32" else np.float64)
        vd = torch.from_numpy(vr).cuda()
        plan.set_potential(vd)
        cr = c.astype(np.complex64 if prec == "fp32" else np.complex128)
        x = torch.from_numpy(cr.reshape(-1)).cuda()
        out = torch.empty_like(x)
        plan.execute(x, out)
        torch.cuda.synchronize()
        want = oracle.apply_potential(g, cr.astype(np.complex128), vr.astype(np.float64), n)
        assert relerr(out.cpu().numpy(), want) <= tol, prec


def test_multik_96_roundtrip(F):
    """96^3, 8 k-points (k ~ U[-0.5,0.5)^3), |G+k| <= 24, 16..128 bands each, one plan."""
    import torch
    n, r = (96, 96, 96), 24.0
    ks = fi.kshifts(8, 3)
    bands = fi.band_counts(8, 16, 128, 3)
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, kshift=ks, bands=bands)
    gs = [plan.sphere(k) for k in range(8)]
    for k in (0, 5):
        assert np.array_equal(gs[k], oracle.sphere_gvectors(n, r, ks[k]))
    parts = [fi.complex_gaussian((int(b), len(g)), 300 + k).astype(np.complex64)
             for k, (g, b) in enumerate(zip(gs, bands))]
    x = torch.from_numpy(np.concatenate([p.reshape(-1) for p in parts])).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    xs = x.cpu().numpy().astype(np.complex128)
    assert relerr(out.cpu().numpy(), 96 ** 3 * xs) <= 2e-6
    # sampled real-space points of two bands of two k-points
    vol = 96 ** 3
    offs = np.concatenate([[0], np.cumsum(bands)])
    pts = sample_points(n, 12, 9)
    for k in (2, 7):
        b0 = int(offs[k])
        R = cube[b0 * vol:(b0 + 2) * vol].view(2, 96, 96, 96).cpu().numpy().astype(np.complex128)
        want = oracle.g2r_points(gs[k], parts[k][:2].astype(np.complex128), n, pts)
        assert relerr(R[:, pts[:, 2], pts[:, 1], pts[:, 0]], want) <= 2e-6


def test_160_g2r_sampled_fp32(F):
    """160^3, |G| <= 40 (radix-5 lengths), sampled outputs in both directions."""
    import torch
    n, r, bands = (160, 160, 160), 40.0, 4
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 5).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    c64 = c.astype(np.complex128)
    assert relerr(out.cpu().numpy(), 160 ** 3 * c64.reshape(-1)) <= 2e-6
    R = cube.view(bands, 160, 160, 160).cpu().numpy().astype(np.complex128)
    pts = sample_points(n, 16, 11)
    want = oracle.g2r_points(g, c64, n, pts)
    assert relerr(R[:, pts[:, 2], pts[:, 1], pts[:, 0]], want) <= 2e-6
    # r -> G of a random cube at a few sampled G (direct O(N^3) sums)
    p2 = F.Plan(n, "r2g", "fp32", radius=r, bands=[1])
    Rr = fi.complex_gaussian((160, 160, 160), 12).astype(np.complex64)
    xr = torch.from_numpy(Rr.reshape(-1)).cuda()
    o2 = torch.empty(p2.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    p2.execute(xr, o2)
    torch.cuda.synchronize()
    sel = np.random.default_rng(13).choice(len(g), 6, replace=False)
    want = oracle.r2g_points(g[sel], Rr.astype(np.complex128), n)
    assert relerr(o2.cpu().numpy()[sel], want) <= 2e-6


def test_160_fp64_roundtrip_sampled(F):
    """160^3 FP64 (slab planes too large for shared memory: kept in global memory)."""
    import torch
    n, r, bands = (160, 160, 160), 40.0, 2
    plan = F.Plan(n, "roundtrip", "fp64", radius=r, bands=[bands])
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 6)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex128, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    assert relerr(out.cpu().numpy(), 160 ** 3 * c.reshape(-1)) <= 1e-12
    R = cube.view(bands, 160, 160, 160).cpu().numpy()
    pts = sample_points(n, 12, 21)
    want = oracle.g2r_points(g, c, n, pts)
    assert relerr(R[:, pts[:, 2], pts[:, 1], pts[:, 0]], want) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp64", 1e-12), ("mixed", 1e-5)])
def test_256_roundtrip_paper_shape(F, prec, tol):
    """256^3 with sphere diameter 128 (|G| <= 64, 1 097 917 G): the paper's
    single-GPU shape; slab planes of 256 x 129 live in global memory. One band
    against the full oracle, the round trip on two bands."""
    import torch
    n, r, bands = (256, 256, 256), 64.0, 2
    plan = F.Plan(n, "roundtrip", prec, radius=r, bands=[bands])
    assert plan.info["slab_planes_global"] == 1
    g = plan.sphere(0)
    assert len(g) == 1097917
    cd = np.complex128 if prec == "fp64" else np.complex64
    c = fi.complex_gaussian((bands, len(g)), 7).astype(cd)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=x.dtype, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    c64 = c.astype(np.complex128)
    assert relerr(out.cpu().numpy(), 256 ** 3 * c64.reshape(-1)) <= tol
    R0 = cube[: 256 ** 3].view(256, 256, 256).cpu().numpy().astype(np.complex128)
    assert relerr(R0, oracle.g2r(g, c64[0], n)) <= tol


@pytest.mark.parametrize("name", ["sphere64_rt", "sphere96_multik", "sphere128_apply", "sphere160_large",
                                  "sphere256_e2", "sphere64_rt_batchfast"])
def test_bench_workloads_in_their_timed_configuration(F, name, tmp_path, monkeypatch):
    """Every bench workload at its full size, built by bench.py itself
    (autotuned, graph-replayed where the bench replays one): the round trip
    of the whole batch equals N0 N1 N2 times the input, and sampled outputs of
    two bands of the first and last k-point match the oracle's direct sums
    (gathered on the device: the 256^3 cube set is 34 GB)."""
    import torch
    import bench
    monkeypatch.setenv("FFTB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    w = bench.Workload(name)
    plan, _ = bench.make_plan(F, w, "fp32", torch.device("cuda", 0))
    gs = [plan.sphere(k) for k in range(w.nk)]
    parts = w.coefficients(gs)
    x = torch.from_numpy(np.concatenate([(p.T if w.layout else p).reshape(-1) for p in parts])
                         .astype(np.complex64)).cuda()
    out = torch.empty_like(x)
    cube = None
    if w.direction == "roundtrip":
        cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    for _ in range(2):  # the second run replays the recorded graph where there is one
        plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()
    vol = w.n[0] * w.n[1] * w.n[2]
    if w.direction == "roundtrip":
        err = (torch.linalg.vector_norm(out - vol * x) / torch.linalg.vector_norm(vol * x)).item()
        assert err <= 2e-6
    sph0 = np.concatenate([[0], np.cumsum([b * len(g) for b, g in zip(w.bands, gs)])])
    band0 = np.concatenate([[0], np.cumsum(w.bands)])
    pts = sample_points(w.n, 8, 31)
    lin = (pts[:, 2] * w.n[1] + pts[:, 1]) * w.n[0] + pts[:, 0]
    for k in sorted({0, w.nk - 1}):
        g, b = gs[k], w.bands[k]
        sel = np.array([0, b - 1])
        c = parts[k][sel].astype(np.complex64).astype(np.complex128)
        if w.direction == "apply":
            v = w.potential().astype(np.float32).astype(np.float64)
            got = out[int(sph0[k]):int(sph0[k + 1])].view(b, len(g))[torch.from_numpy(sel).cuda()].cpu().numpy()
            assert relerr(got, oracle.apply_potential(g, c, v, w.n)) <= 2e-6
            continue
        if w.layout:  # [N2][N1][N0][B] per k-point
            idx = band0[k] * vol + lin[None, :] * b + sel[:, None]
        else:         # [B][N2][N1][N0]
            idx = (band0[k] + sel[:, None]) * vol + lin[None, :]
        got = cube[torch.from_numpy(idx.reshape(-1).astype(np.int64)).cuda()].cpu().numpy().reshape(2, -1)
        assert relerr(got, oracle.g2r_points(g, c, w.n, pts)) <= 2e-6
    del cube, out, x, plan
    torch.cuda.empty_cache()
