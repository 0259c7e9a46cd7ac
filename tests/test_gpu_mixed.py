"""The split-precision tensor-core precision (MIXED_TC) against the FP64
oracle at the full workload shapes, relative L2 <= 1e-5: the fused V(r)
apply at 128^3, the round trip with 8 k-points at 96^3, and 160^3 (lengths
with radix-3 and radix-5 factors). Whole bands are compared where the oracle
finishes in seconds; larger outputs on samples the oracle computes one by one
(direct sums)."""
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


def sample_points(n, count, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, n[0], count), rng.integers(0, n[1], count),
                     rng.integers(0, n[2], count)], axis=1)


def test_mixed_apply_128_vs_oracle(F):
    """128^3, |G| <= 32, V = 32 Gaussians of width 4, 8 bands: the fused
    apply kernel of the MIXED_TC precision against the full oracle."""
    import torch
    n, r, bands = (128, 128, 128), 32.0, 8
    v = fi.gaussian_potential(n, 32, 4.0, seed=4).astype(np.float32)
    plan = F.Plan(n, "apply", "mixed", radius=r, bands=[bands])
    g = plan.sphere(0)
    assert len(g) == 137065
    plan.set_potential(torch.from_numpy(v).cuda())
    c = fi.complex_gaussian((bands, len(g)), 4).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    plan.execute(x, out)
    torch.cuda.synchronize()
    plan.check()
    want = oracle.apply_potential(g, c.astype(np.complex128), v.astype(np.float64), n)
    got = out.cpu().numpy().reshape(bands, -1)
    assert relerr(got, want) <= TOL
    # each band on its own as well (a band much smaller than the rest would
    # hide in the batch norm)
    for b in range(bands):
        assert relerr(got[b], want[b]) <= TOL, b


def test_mixed_multik_96_vs_oracle(F):
    """96^3, 8 k-points k ~ U[-0.5,0.5)^3, |G+k| <= 24, uneven bands per
    k-point, one plan: the round trip of every band, the real-space cube of
    two bands of three k-points at sampled points, one band against the full
    oracle, and r -> G of random cubes at sampled G."""
    import torch
    n, r = (96, 96, 96), 24.0
    ks = fi.kshifts(8, 3)
    bands = [3, 1, 2, 4, 1, 2, 3, 2]
    plan = F.Plan(n, "roundtrip", "mixed", radius=r, kshift=ks, bands=bands)
    gs = [plan.sphere(k) for k in range(8)]
    for k in range(8):
        assert np.array_equal(gs[k], oracle.sphere_gvectors(n, r, ks[k]))
    parts = [fi.complex_gaussian((b, len(g)), 400 + k).astype(np.complex64)
             for k, (g, b) in enumerate(zip(gs, bands))]
    x = torch.from_numpy(np.concatenate([p.reshape(-1) for p in parts])).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()
    xs = x.cpu().numpy().astype(np.complex128)
    assert relerr(out.cpu().numpy(), 96 ** 3 * xs) <= TOL
    vol = 96 ** 3
    offs = np.concatenate([[0], np.cumsum(bands)])
    pts = sample_points(n, 16, 19)
    for k in (0, 3, 7):
        b0, nb = int(offs[k]), bands[k]
        R = cube[b0 * vol:(b0 + nb) * vol].view(nb, 96, 96, 96).cpu().numpy().astype(np.complex128)
        want = oracle.g2r_points(gs[k], parts[k].astype(np.complex128), n, pts)
        assert relerr(R[:, pts[:, 2], pts[:, 1], pts[:, 0]], want) <= TOL
        if k == 3:
            assert relerr(R[0], oracle.g2r(gs[k], parts[k][0].astype(np.complex128), n)) <= TOL
    # r -> G of random cubes (one band per k-point)
    p2 = F.Plan(n, "r2g", "mixed", radius=r, kshift=ks, bands=[1] * 8)
    Rr = fi.complex_gaussian((8, 96, 96, 96), 410).astype(np.complex64)
    xr = torch.from_numpy(Rr.reshape(-1)).cuda()
    o2 = torch.empty(p2.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    p2.execute(xr, o2)
    torch.cuda.synchronize()
    got = o2.cpu().numpy()
    off = 0
    for k in range(8):
        g = gs[k]
        if k in (1, 6):
            sel = np.random.default_rng(420 + k).choice(len(g), 5, replace=False)
            want = oracle.r2g_points(g[sel], Rr[k].astype(np.complex128), n)
            assert relerr(got[off + sel], want) <= TOL
        if k == 2:
            want = oracle.r2g(g, Rr[k].astype(np.complex128), n)
            assert relerr(got[off:off + len(g)], want) <= TOL
        off += len(g)


def test_mixed_160_vs_oracle(F):
    """160^3, |G| <= 40, MIXED_TC: round trip of 4 bands, the cube of every
    band at sampled points, one whole band against the full oracle, and r -> G
    of a random cube at sampled G."""
    import torch
    n, r, bands = (160, 160, 160), 40.0, 4
    plan = F.Plan(n, "roundtrip", "mixed", radius=r, bands=[bands])
    g = plan.sphere(0)
    assert len(g) == 267761
    c = fi.complex_gaussian((bands, len(g)), 5).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()
    c64 = c.astype(np.complex128)
    assert relerr(out.cpu().numpy(), 160 ** 3 * c64.reshape(-1)) <= TOL
    R = cube.view(bands, 160, 160, 160).cpu().numpy().astype(np.complex128)
    pts = sample_points(n, 16, 23)
    want = oracle.g2r_points(g, c64, n, pts)
    assert relerr(R[:, pts[:, 2], pts[:, 1], pts[:, 0]], want) <= TOL
    assert relerr(R[1], oracle.g2r(g, c64[1], n)) <= TOL
    p2 = F.Plan(n, "r2g", "mixed", radius=r, bands=[1])
    Rr = fi.complex_gaussian((160, 160, 160), 24).astype(np.complex64)
    xr = torch.from_numpy(Rr.reshape(-1)).cuda()
    o2 = torch.empty(p2.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    p2.execute(xr, o2)
    torch.cuda.synchronize()
    sel = np.random.default_rng(25).choice(len(g), 6, replace=False)
    want = oracle.r2g_points(g[sel], Rr.astype(np.complex128), n)
    assert relerr(o2.cpu().numpy()[sel], want) <= TOL


@pytest.mark.parametrize("name", ["sphere128_apply", "sphere160_large"])
def test_mixed_bench_workloads_in_their_timed_configuration(F, name, tmp_path, monkeypatch):
    """The MIXED_TC plan the benchmark times beside FP32, built by bench.py
    (autotuned), at the workload's full size: round trip of the whole batch
    (or the apply of two bands) against N0 N1 N2 x the input (the oracle)."""
    import torch
    import bench
    monkeypatch.setenv("FFTB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    w = bench.Workload(name)
    plan, _ = bench.make_plan(F, w, "mixed", torch.device("cuda", 0))
    gs = [plan.sphere(k) for k in range(w.nk)]
    parts = w.coefficients(gs)
    x = torch.from_numpy(np.concatenate([p.reshape(-1) for p in parts]).astype(np.complex64)).cuda()
    out = torch.empty_like(x)
    cube = None
    if w.direction == "roundtrip":
        cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()
    vol = w.n[0] * w.n[1] * w.n[2]
    if w.direction == "roundtrip":
        err = (torch.linalg.vector_norm(out - vol * x) / torch.linalg.vector_norm(vol * x)).item()
        assert err <= TOL
        pts = sample_points(w.n, 6, 41)
        lin = torch.from_numpy((pts[:, 2] * w.n[1] + pts[:, 1]) * w.n[0] + pts[:, 0]).cuda()
        b = w.bands[0] - 1
        got = cube[b * vol:(b + 1) * vol][lin].cpu().numpy()
        want = oracle.g2r_points(gs[0], parts[0][b].astype(np.complex64).astype(np.complex128), w.n, pts)
        assert relerr(got, want) <= TOL
    else:
        g = gs[0]
        v = w.potential().astype(np.float32).astype(np.float64)
        got = out[: 2 * len(g)].cpu().numpy().reshape(2, -1)
        c = parts[0][:2].astype(np.complex64).astype(np.complex128)
        assert relerr(got, oracle.apply_potential(g, c, v, w.n)) <= TOL
    del cube, out, x, plan
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,r,direction", [((128, 128, 128), 32.0, "apply"), ((64, 64, 64), 16.0, "roundtrip")])
def test_mixed_tensor_cores_on_and_off(F, n, r, direction, tmp_path, monkeypatch):
    """MIXED_TC plans that have tensor-core kernels (mma.sync radix-8 passes
    at 128, tcgen05 plane products at 64): each setting of
    fftb_plan_set_tensor_cores against the oracle and in the plan's info, then
    the autotuner's choice between them, recorded in its cache line."""
    import torch
    monkeypatch.setenv("FFTB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    bands = 3
    plan = F.Plan(n, direction, "mixed", radius=r, bands=[bands])
    assert plan.info["tensor_cores_available"] == 1
    used = plan.info["tensor_core_passes"] | plan.info["tensor_core_planes"]
    assert used != 0
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 61).astype(np.complex64)
    c64 = c.astype(np.complex128)
    if direction == "apply":
        v = fi.gaussian_potential(n, 16, 4.0, seed=62).astype(np.float32)
        plan.set_potential(torch.from_numpy(v).cuda())
        want = oracle.apply_potential(g, c64, v.astype(np.float64), n)
    else:
        want = np.prod(n) * c64
        cube0 = oracle.g2r(g, c64[0], n)
    x = torch.from_numpy(c.reshape(-1)).cuda()

    def run():
        out = torch.empty_like(x)
        cube = None
        if direction == "roundtrip":
            cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
        plan.execute(x, out, cube)
        torch.cuda.synchronize()
        plan.check()
        got = out.cpu().numpy().reshape(bands, -1)
        for b in range(bands):
            assert relerr(got[b], want[b]) <= TOL, b
        if cube is not None:
            R0 = cube[:np.prod(n)].view(n[2], n[1], n[0]).cpu().numpy().astype(np.complex128)
            assert relerr(R0, cube0) <= TOL

    run()
    plan.set_tensor_cores(False)
    assert plan.info["tensor_core_passes"] == 0 and plan.info["tensor_core_planes"] == 0
    assert plan.info["tensor_cores_available"] == 1
    run()
    plan.set_tensor_cores(True)
    assert plan.info["tensor_core_passes"] | plan.info["tensor_core_planes"] == used
    run()
    plan.autotune(2)
    line = (tmp_path / "tune.txt").read_text().strip().split()
    assert len(line) == 14 and line[-2] in ("0", "1") and line[-1] == "0"  # ..., tensor cores, clusters
    assert (line[-2] == "1") == ((plan.info["tensor_core_passes"] | plan.info["tensor_core_planes"]) != 0)
    run()


def test_mixed_tensor_core_switch_where_none_exist(F):
    """A MIXED_TC plan with no tensor-core stage (160 has no radix-8 pass):
    the switch is a no-op; FP32 and FP64 plans reject it."""
    p = F.Plan((160, 160, 160), "g2r", "mixed", radius=40.0, bands=[1])
    assert p.info["tensor_cores_available"] == 0 and p.info["tensor_core_passes"] == 0
    p.set_tensor_cores(True)
    p.set_tensor_cores(False)
    assert p.info["tensor_core_passes"] == 0 and p.info["tensor_core_planes"] == 0
    for prec in ("fp32", "fp64"):
        q = F.Plan((64, 64, 64), "g2r", prec, radius=16.0, bands=[1])
        assert q.info["tensor_cores_available"] == 0
        with pytest.raises(F.FFTBError) as e:
            q.set_tensor_cores(True)
        assert e.value.status == F.FFTB_ERR_UNSUPPORTED


def test_mixed_batch_fastest_groups_with_tensor_cores_off(F):
    """A batch-fastest MIXED_TC plan at 64^3: with the tensor cores on the
    plane stages run one band per plane (the grouped kernels are FP32), with
    them off the grouped FP32 kernels; both against the oracle."""
    import torch
    n, r, bands = (64, 64, 64), 16.0, 6
    plan = F.Plan(n, "g2r", "mixed", radius=r, bands=[bands], layout=1)
    assert plan.info["tensor_cores_available"] == 1 and plan.info["plane_band_group"] == 0
    with pytest.raises(F.FFTBError) as e:
        plan.set_band_groups(True)
    assert e.value.status == F.FFTB_ERR_UNSUPPORTED
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 63).astype(np.complex64)
    want = np.moveaxis(oracle.g2r(g, c.astype(np.complex128), n), 0, -1)  # [N2][N1][N0][B]
    x = torch.from_numpy(np.ascontiguousarray(c.T).reshape(-1)).cuda()
    for tc in (True, False):
        plan.set_tensor_cores(tc)
        assert plan.info["plane_band_group"] == (0 if tc else 4)
        out = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
        plan.execute(x, out)
        torch.cuda.synchronize()
        plan.check()
        assert relerr(out.cpu().numpy().reshape(want.shape), want) <= TOL, tc
