"""The generic-extent path (extents outside the compiled list, N0 != N1,
any extent whose prime factors are 2, 3 and 5: the cuboid grids of Sec. 3.2 /
Fig. 5 with the plane-wave sphere of Sec. 2.2) against the FP64 oracle:
non-square and odd grids, listed lengths with N0 != N1, k-points with uneven
band counts split into chunks, an explicit sphere order, the batch-fastest
layout, the fused V(r) apply, and a large grid on sampled outputs."""
import numpy as np
import pytest

import fftb_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6, "mixed": 2e-6}


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


def cdt(prec):
    return np.complex128 if prec == "fp64" else np.complex64


def run(F, plan, x, out_elems, cube=False):
    import torch
    td = torch.complex128 if plan.precision == F.FFTB_FP64 else torch.complex64
    xd = torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).to(td).cuda()
    out = torch.empty(out_elems, dtype=td, device="cuda")
    cb = torch.empty(plan.info["cube_elems"], dtype=td, device="cuda") if cube else None
    plan.execute(xd, out, cb)
    torch.cuda.synchronize()
    plan.check()
    return out.cpu().numpy().astype(np.complex128), (None if cb is None else cb.cpu().numpy().astype(np.complex128))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("n,r,k", [((72, 80, 90), 17.5, (0.2, -0.35, 0.1)),
                                   ((15, 27, 25), 5.0, None),
                                   ((64, 96, 48), 11.0, (0.0, 0.4, -0.2)),
                                   ((100, 36, 54), 12.0, None)])
def test_generic_g2r_r2g_roundtrip_vs_oracle(F, n, r, k, prec):
    bands = 3
    kv = k if k else (0.0, 0.0, 0.0)
    g = oracle.sphere_gvectors(n, r, kv)
    kw = dict(radius=r, bands=[bands])
    if k:
        kw["kshift"] = [k]
    c = fi.complex_gaussian((bands, len(g)), 501).astype(cdt(prec)).astype(np.complex128)
    vol = n[0] * n[1] * n[2]
    p1 = F.Plan(n, "g2r", prec, **kw)
    assert p1.info["generic_path"] == 1 and p1.info["tensor_core_passes"] == 0
    assert p1.info["kernels_per_execute"] == 3 * -(-bands // p1.info["chunk_bands"])
    assert np.array_equal(p1.sphere(0), g)
    cube, _ = run(F, p1, c, p1.info["cube_elems"])
    assert relerr(cube, oracle.g2r(g, c, n).reshape(-1)) <= TOL[prec]
    R = fi.complex_gaussian((bands, n[2], n[1], n[0]), 502).astype(cdt(prec)).astype(np.complex128)
    p2 = F.Plan(n, "r2g", prec, **kw)
    sph, _ = run(F, p2, R, p2.info["sphere_elems"])
    assert relerr(sph, oracle.r2g(g, R, n).reshape(-1)) <= TOL[prec]
    p3 = F.Plan(n, "roundtrip", prec, **kw)
    back, cb = run(F, p3, c, p3.info["sphere_elems"], cube=True)
    assert relerr(cb, oracle.g2r(g, c, n).reshape(-1)) <= TOL[prec]
    assert relerr(back, vol * c.reshape(-1)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_generic_apply_vs_oracle(F, prec):
    import torch
    n, r, bands = (72, 80, 90), 17.5, 3
    g = oracle.sphere_gvectors(n, r)
    v = fi.gaussian_potential(n, 8, 4.0, seed=503).astype(np.float64 if prec == "fp64" else np.float32)
    plan = F.Plan(n, "apply", prec, radius=r, bands=[bands])
    plan.set_potential(torch.from_numpy(v).cuda())
    c = fi.complex_gaussian((bands, len(g)), 504).astype(cdt(prec)).astype(np.complex128)
    out, _ = run(F, plan, c, plan.info["sphere_elems"])
    assert plan.info["kernels_per_execute"] == 5 * -(-bands // plan.info["chunk_bands"])
    assert relerr(out, oracle.apply_potential(g, c, v.astype(np.float64), n)) <= TOL[prec]


def test_generic_multik_chunks_explicit_order_and_layout(F):
    """Three k-points with 2, 0 and 5 bands in chunks of 2 (chunks straddle
    k-points); then a permuted explicit sphere list; then the batch-fastest
    layout, equal to the band-major results permuted."""
    n, r = (40, 45, 36), 8.5
    ks = [(0.1, 0.2, -0.3), (-0.4, 0.0, 0.25), (0.3, -0.45, 0.0)]
    bands = [2, 0, 5]
    gs = [oracle.sphere_gvectors(n, r, k) for k in ks]
    parts = [fi.complex_gaussian((b, len(g)), 510 + i) for i, (g, b) in enumerate(zip(gs, bands))]
    x = np.concatenate([p.reshape(-1) for p in parts])
    plan = F.Plan(n, "g2r", "fp64", radius=r, kshift=ks, bands=bands, max_chunk_bands=2)
    assert plan.info["chunk_bands"] == 2
    cube, _ = run(F, plan, x, plan.info["cube_elems"])
    want = np.concatenate([oracle.g2r(g, p, n).reshape(-1) for g, p in zip(gs, parts) if len(p)])
    assert relerr(cube, want) <= 1e-12
    # explicit order
    perm = np.random.default_rng(511).permutation(len(gs[2]))
    gu = gs[2][perm]
    pe = F.Plan(n, "roundtrip", "fp64", g_lists=[gu], bands=[2])
    cu = fi.complex_gaussian((2, len(gu)), 512)
    back, cb = run(F, pe, cu, pe.info["sphere_elems"], cube=True)
    assert relerr(cb, oracle.g2r(gu, cu, n).reshape(-1)) <= 1e-12
    assert relerr(back, np.prod(n) * cu.reshape(-1)) <= 1e-12
    # batch-fastest: sphere [ngw][B], cube [N2][N1][N0][B]
    g = gs[0]
    cb2 = fi.complex_gaussian((4, len(g)), 513)
    pb = F.Plan(n, "g2r", "fp64", radius=r, kshift=[ks[0]], bands=[4], layout=1)
    cube_b, _ = run(F, pb, cb2.T, pb.info["cube_elems"])
    want = oracle.g2r(g, cb2, n)  # [B][N2][N1][N0]
    assert relerr(cube_b.reshape(n[2], n[1], n[0], 4), np.moveaxis(want, 0, -1)) <= 1e-12


def test_generic_large_grid_sampled(F):
    """A 320 x 288 x 240 grid (none of the extents compiled), |G| <= 60, FP32:
    sampled real-space points of each band against direct sums, the round trip
    against N0 N1 N2 times the input, and r -> G of a random cube at sampled G."""
    import torch
    n, r, bands = (320, 288, 240), 60.0, 2
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    assert plan.info["generic_path"] == 1
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 520).astype(np.complex64)
    back, cube = run(F, plan, c, plan.info["sphere_elems"], cube=True)
    c64 = c.astype(np.complex128)
    assert relerr(back, np.prod(n) * c64.reshape(-1)) <= 2e-6
    rng = np.random.default_rng(521)
    pts = np.stack([rng.integers(0, n[d], 12) for d in range(3)], axis=1)
    R = cube.reshape(bands, n[2], n[1], n[0])
    assert relerr(R[:, pts[:, 2], pts[:, 1], pts[:, 0]], oracle.g2r_points(g, c64, n, pts)) <= 2e-6
    p2 = F.Plan(n, "r2g", "fp32", radius=r, bands=[1])
    Rr = fi.complex_gaussian((n[2], n[1], n[0]), 522).astype(np.complex64)
    sph, _ = run(F, p2, Rr, p2.info["sphere_elems"])
    sel = rng.choice(len(g), 5, replace=False)
    assert relerr(sph[sel], oracle.r2g_points(g[sel], Rr.astype(np.complex128), n)) <= 2e-6
    del cube, R
    torch.cuda.empty_cache()


def test_generic_setters(F):
    plan = F.Plan((72, 80, 90), "roundtrip", "fp32", radius=17.5, bands=[2])
    plan.autotune(2)  # one kernel per stage: nothing to choose, results unchanged
    for fn in (lambda: plan.set_prefetch(1), lambda: plan.set_slab_buffers(2), lambda: plan.set_radix_schedule(1, 0),
               lambda: plan.set_band_groups(True)):
        with pytest.raises(F.FFTBError) as e:
            fn()
        assert e.value.status == F.FFTB_ERR_UNSUPPORTED
