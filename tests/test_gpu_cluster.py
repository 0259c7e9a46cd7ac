"""The 256-point plane stages on two-CTA clusters (each CTA holds half of the
slab plane in shared memory, the y outputs of the other half go to its
partner's shared memory) against the FP64 oracle: the E2 sphere (|G| <= 64,
129 slabs) in G -> r, r -> G, round trip and the fused apply; two k-points
with uneven bands in chunks that straddle them, one sphere with a gap in a
column; the batch-fastest layout; the switch, the info fields and the
autotuner's choice."""
import numpy as np
import pytest

import fftb_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

N = (256, 256, 256)
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
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_cluster_roundtrip_and_r2g_vs_oracle(F):
    import torch
    r, bands = 64.0, 2
    plan = F.Plan(N, "roundtrip", "fp32", radius=r, bands=[bands])
    assert plan.info["plane_clusters"] == 8  # available, not in use by default
    plan.set_plane_clusters(True)
    assert plan.info["plane_clusters"] == 15 and plan.info["slab_planes_global"] == 0
    assert plan.info["prefetch"] == 0
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 701).astype(np.complex64)
    c64 = c.astype(np.complex128)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()
    vol = np.prod(N)
    assert relerr(out.cpu().numpy(), vol * c64.reshape(-1)) <= TOL
    R = cube.view(bands, 256, 256, 256)
    assert relerr(R[1].cpu().numpy(), oracle.g2r(g, c64[1], N)) <= TOL
    # the single-CTA kernels (slab planes in global memory) agree
    ref = cube.clone()
    plan.set_plane_clusters(False)
    assert plan.info["plane_clusters"] == 8 and plan.info["slab_planes_global"] == 1
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    assert (torch.linalg.vector_norm(cube - ref) / torch.linalg.vector_norm(ref)).item() <= TOL
    del R, ref, cube
    # r -> G of a random cube at sampled G
    p2 = F.Plan(N, "r2g", "fp32", radius=r, bands=[1])
    p2.set_plane_clusters(True)
    Rr = fi.complex_gaussian((256, 256, 256), 702).astype(np.complex64)
    o2 = torch.empty(p2.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    p2.execute(torch.from_numpy(Rr.reshape(-1)).cuda(), o2)
    torch.cuda.synchronize()
    p2.check()
    sel = np.random.default_rng(703).choice(len(g), 8, replace=False)
    assert relerr(o2.cpu().numpy()[sel], oracle.r2g_points(g[sel], Rr.astype(np.complex128), N)) <= TOL
    torch.cuda.empty_cache()


def test_cluster_apply_vs_oracle(F):
    import torch
    r = 64.0
    v = fi.gaussian_potential(N, 16, 6.0, seed=704).astype(np.float32)
    plan = F.Plan(N, "apply", "fp32", radius=r, bands=[1])
    plan.set_plane_clusters(True)
    plan.set_potential(torch.from_numpy(v).cuda())
    g = plan.sphere(0)
    c = fi.complex_gaussian((1, len(g)), 705).astype(np.complex64)
    out = torch.empty(plan.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(torch.from_numpy(c.reshape(-1)).cuda(), out)
    torch.cuda.synchronize()
    plan.check()
    want = oracle.apply_potential(g, c.astype(np.complex128), v.astype(np.float64), N)
    assert relerr(out.cpu().numpy(), want) <= TOL


def test_cluster_kpoints_gap_and_batch_fastest(F):
    """Two k-points (one sphere shifted, one with the stick (x, y) = (3, 0)
    taken out, so its columns are indexed through the scratch rows) with 1 and
    2 bands in chunks of 2; then the batch-fastest layout of 3 bands."""
    import torch
    r = 40.0
    g0 = oracle.sphere_gvectors(N, r, (0.25, -0.1, 0.3))
    g1 = oracle.sphere_gvectors(N, r)
    g1 = g1[~((g1[:, 0] == 3) & (g1[:, 1] == 0))]
    plan = F.Plan(N, "g2r", "fp32", g_lists=[g0, g1], bands=[1, 2], max_chunk_bands=2)
    plan.set_plane_clusters(True)
    c = [fi.complex_gaussian((1, len(g0)), 706), fi.complex_gaussian((2, len(g1)), 707)]
    c = [a.astype(np.complex64) for a in c]
    x = torch.from_numpy(np.concatenate([a.reshape(-1) for a in c])).cuda()
    out = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out)
    torch.cuda.synchronize()
    plan.check()
    got = out.view(3, 256, 256, 256)
    assert relerr(got[0].cpu().numpy(), oracle.g2r(g0, c[0][0].astype(np.complex128), N)) <= TOL
    assert relerr(got[2].cpu().numpy(), oracle.g2r(g1, c[1][1].astype(np.complex128), N)) <= TOL
    del got, out
    # r -> G of the same k-points from random cubes, at sampled G
    p2 = F.Plan(N, "r2g", "fp32", g_lists=[g0, g1], bands=[1, 2], max_chunk_bands=2)
    p2.set_plane_clusters(True)
    R = fi.complex_gaussian((3, 256, 256, 256), 708).astype(np.complex64)
    o2 = torch.empty(p2.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    p2.execute(torch.from_numpy(R.reshape(-1)).cuda(), o2)
    torch.cuda.synchronize()
    p2.check()
    o2 = o2.cpu().numpy()
    rng = np.random.default_rng(709)
    s0 = rng.choice(len(g0), 5, replace=False)
    s1 = rng.choice(len(g1), 5, replace=False)
    assert relerr(o2[:len(g0)][s0], oracle.r2g_points(g0[s0], R[0].astype(np.complex128), N)) <= TOL
    b2 = o2[len(g0) + len(g1):]
    assert relerr(b2[s1], oracle.r2g_points(g1[s1], R[2].astype(np.complex128), N)) <= TOL
    del R
    # batch-fastest: sphere [ngw][B], cube [N2][N1][N0][B]
    pb = F.Plan(N, "g2r", "fp32", radius=r, bands=[3], layout=1)
    pb.set_plane_clusters(True)
    g = pb.sphere(0)
    cb = fi.complex_gaussian((3, len(g)), 710).astype(np.complex64)
    ob = torch.empty(pb.info["cube_elems"], dtype=torch.complex64, device="cuda")
    pb.execute(torch.from_numpy(np.ascontiguousarray(cb.T).reshape(-1)).cuda(), ob)
    torch.cuda.synchronize()
    pb.check()
    band1 = ob.view(256, 256, 256, 3)[..., 1].cpu().numpy()
    assert relerr(band1, oracle.g2r(g, cb[1].astype(np.complex128), N)) <= TOL
    torch.cuda.empty_cache()


def test_cluster_switch_and_autotune(F, tmp_path, monkeypatch):
    import torch
    monkeypatch.setenv("FFTB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    p64 = F.Plan(N, "g2r", "fp64", radius=64.0, bands=[1])
    assert p64.info["plane_clusters"] == 0
    with pytest.raises(F.FFTBError) as e:
        p64.set_plane_clusters(True)
    assert e.value.status == F.FFTB_ERR_UNSUPPORTED
    q = F.Plan((128, 128, 128), "g2r", "fp32", radius=32.0, bands=[1])
    assert q.info["plane_clusters"] == 0
    plan = F.Plan(N, "roundtrip", "fp32", radius=64.0, bands=[4])
    plan.autotune(1)
    line = (tmp_path / "tune.txt").read_text().strip().split()
    # the stages on clusters (bit 0 G->r, bit 1 r->G), as chosen per stage and as the plan reports them
    assert len(line) == 14 and 0 <= int(line[-1]) <= 3 and int(line[-1]) == plan.info["plane_clusters"] & 7
    g = plan.sphere(0)
    c = fi.complex_gaussian((4, len(g)), 711).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()
    assert relerr(out.cpu().numpy(), np.prod(N) * c.astype(np.complex128).reshape(-1)) <= TOL
    del cube
    torch.cuda.empty_cache()
